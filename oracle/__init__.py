"""CPU oracle for BGV encrypted comparison.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
statement of what the CUDA path computes.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.  The
product package never imports it, and the two share no code: the only module
both sides use is the seeded input generator, which holds none of the method's
arithmetic.

Layout
  bgv_oracle.c  ring arithmetic, NTT, keys, key switching, modulus switching
                (exact u128 arithmetic, plain definitions)
  bgv.py        ctypes wrapper and ciphertext bookkeeping (levels)
  encoding.py   the slot structure of F_p-valued plaintexts in X^N+1
  ltpoly.py     the univariate less-than polynomial over Z_p
  circuits.py   Paterson-Stockmeyer evaluation, digit merge, LT/EQ/max/min

What is pinned, and by what, is listed in the header of each module.
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "bgv_oracle.c")


def build(force: bool = False) -> str:
    """Compile bgv_oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


def _declare(L):
    u64, i64, ci, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    sig = {
        "orc_mulmod": (u64, [u64, u64, u64]),
        "orc_powmod": (u64, [u64, u64, u64]),
        "orc_is_prime": (ci, [u64]),
        "orc_find_primes": (ci, [u64, u64, u64, ci, vp]),
        "orc_smallest_generator": (u64, [u64]),
        "orc_ctx_new": (vp, [ci, u64, ci, ci, u64, u64, u64]),
        "orc_ctx_free": (None, [vp]),
        "orc_ctx_primes": (None, [vp, vp]),
        "orc_ctx_psi": (u64, [vp, ci]),
        "orc_ntt_direct": (None, [vp, ci, vp, vp]),
        "orc_ntt": (None, [vp, ci, vp]),
        "orc_intt": (None, [vp, ci, vp]),
        "orc_polymul": (None, [vp, ci, vp, vp, vp]),
        "orc_polymul_int": (None, [vp, vp, vp, vp]),
        "orc_automorphism_int": (None, [vp, vp, u64, vp]),
        "orc_automorphism": (None, [vp, vp, ci, ci, u64, vp]),
        "orc_add": (None, [vp, vp, vp, ci, ci, vp]),
        "orc_sub": (None, [vp, vp, vp, ci, ci, vp]),
        "orc_neg": (None, [vp, vp, ci, ci, vp]),
        "orc_mul_const": (None, [vp, vp, i64, ci, ci, vp]),
        "orc_add_const": (None, [vp, vp, i64, ci, vp]),
        "orc_tensor": (None, [vp, vp, vp, ci, vp]),
        "orc_keygen": (None, [vp, vp, vp, vp, vp]),
        "orc_encrypt": (None, [vp, vp, vp, vp, vp, vp, vp]),
        "orc_dot_sk": (None, [vp, vp, ci, vp, vp]),
        "orc_dnum": (ci, [vp, ci]),
        "orc_ksk_gen": (None, [vp, vp, vp, vp, vp, vp]),
        "orc_fbc": (None, [vp, vp, vp, ci, vp, ci, vp]),
        "orc_keyswitch": (None, [vp, vp, ci, vp, vp]),
        "orc_relin": (None, [vp, vp, ci, vp, vp]),
        "orc_rotate": (None, [vp, vp, ci, u64, vp, vp]),
        "orc_modswitch": (None, [vp, vp, ci, ci, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
