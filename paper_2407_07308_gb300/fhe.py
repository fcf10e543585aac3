"""Python binding of libfhe_gb300.so (the C ABI in include/fhe.h).

Argument marshalling only: every function here converts numpy arrays and
handles to C arguments, calls the C function of the same name and raises
FheError on a negative return code.  All computation happens in the CUDA
library.  PyTorch provides device memory (its caching allocator, handed to the
library as an allocator vtable) and the CUDA stream.

The library must have been built (``paper_2407_07308_gb300.build.build()``);
importing this module on a machine without it raises immediately -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_int, c_int32, c_int64, c_size_t, c_uint64,
                    c_void_p)

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfhe_gb300.so")

ERRORS = {
    -1: "FHE_EINVAL", -2: "FHE_EMISMATCH", -3: "FHE_ELEVEL", -4: "FHE_ENOMEM", -5: "FHE_EBUDGET",
    -6: "FHE_ETIMEOUT", -7: "FHE_ECUDA", -8: "FHE_ENOKEY", -9: "FHE_EUNSUPPORTED",
}
OPS = {1: "mul", 2: "add", 3: "sub", 4: "cmul", 5: "cadd", 6: "neg", 7: "rot", 8: "padd", 9: "psub", 10: "pmul"}


class FheError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class fhe_params(Structure):
    _fields_ = [("log_n", c_int), ("p", c_uint64), ("L", c_int), ("K", c_int), ("prime_mod", c_uint64),
                ("prime_lo", c_uint64), ("prime_hi", c_uint64)]


ALLOC_FN = CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class fhe_allocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


class fhe_server_config(Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_batch", c_int), ("batch_flags", c_int)]


class fhe_request_info(Structure):
    _fields_ = [("state", c_int), ("error", c_int), ("t_submit_ms", ctypes.c_double),
                ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double), ("est_bytes", ctypes.c_uint64)]


class fhe_server_status(Structure):
    _fields_ = [("queued", ctypes.c_longlong), ("running", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("batches", ctypes.c_longlong), ("admitted_bytes", ctypes.c_uint64),
                ("admitted_peak_bytes", ctypes.c_uint64)]


FHE_REQ_QUEUED, FHE_REQ_RUNNING, FHE_REQ_DONE = 0, 1, 2


class fhe_job(Structure):
    _fields_ = [("ctx", c_void_p), ("evk", c_void_p), ("kind", c_int), ("d", c_int), ("x", c_void_p),
                ("y", c_void_p), ("out0", c_void_p), ("out1", c_void_p)]


FHE_JOB_COMPARE, FHE_JOB_MAXMIN, FHE_JOB_SORT = 1, 2, 3


class fhe_info(Structure):
    _fields_ = [("N", c_int), ("L", c_int), ("K", c_int), ("slots", c_int), ("subring", c_int),
                ("dnum_max", c_int), ("p", c_uint64)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2407_07308_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, ci, u64, i64 = c_void_p, c_int, c_uint64, c_int64
        sig = {
            "fhe_ctx_create": (ci, [POINTER(fhe_params), POINTER(fhe_allocator), vp, POINTER(vp)]),
            "fhe_ctx_destroy": (None, [vp]),
            "fhe_last_error": (c_char_p, [vp]),
            "fhe_ctx_info": (ci, [vp, POINTER(fhe_info)]),
            "fhe_ctx_primes": (ci, [vp, vp]),
            "fhe_ctx_set_stream": (ci, [vp, vp]),
            "fhe_ctx_sync": (ci, [vp]),
            "fhe_ctx_memory": (ci, [vp, POINTER(u64), POINTER(u64)]),
            "fhe_ctx_set_budget": (ci, [vp, u64]),
            "fhe_ctx_launches": (i64, [vp]),
            "fhe_keygen_explicit": (ci, [vp, vp, vp, vp, POINTER(vp), POINTER(vp)]),
            "fhe_keygen": (ci, [vp, u64, POINTER(vp), POINTER(vp)]),
            "fhe_sk_destroy": (None, [vp]),
            "fhe_pk_destroy": (None, [vp]),
            "fhe_evk_create_explicit": (ci, [vp, vp, vp, ci, vp, vp, POINTER(vp)]),
            "fhe_evk_create": (ci, [vp, vp, vp, ci, u64, POINTER(vp)]),
            "fhe_evk_destroy": (None, [vp]),
            "fhe_encrypt_explicit": (ci, [vp, vp, vp, ci, vp, vp, vp, POINTER(vp)]),
            "fhe_encrypt": (ci, [vp, vp, vp, ci, u64, POINTER(vp)]),
            "fhe_decrypt": (ci, [vp, vp, vp, vp]),
            "fhe_ct_destroy": (None, [vp]),
            "fhe_ct_shape": (ci, [vp, POINTER(ci), POINTER(ci), POINTER(ci)]),
            "fhe_ct_export_coeff": (ci, [vp, vp, vp]),
            "fhe_ct_import_coeff": (ci, [vp, vp, ci, ci, ci, POINTER(vp)]),
            "fhe_ct_load_coeff": (ci, [vp, vp, vp]),
            "fhe_add": (ci, [vp, vp, vp, POINTER(vp)]),
            "fhe_sub": (ci, [vp, vp, vp, POINTER(vp)]),
            "fhe_neg": (ci, [vp, vp, POINTER(vp)]),
            "fhe_mul_const": (ci, [vp, vp, i64, POINTER(vp)]),
            "fhe_add_const": (ci, [vp, vp, i64, POINTER(vp)]),
            "fhe_mul": (ci, [vp, vp, vp, POINTER(vp)]),
            "fhe_relinearize": (ci, [vp, vp, vp, POINTER(vp)]),
            "fhe_mod_switch": (ci, [vp, vp, ci, POINTER(vp)]),
            "fhe_rotate": (ci, [vp, vp, vp, i64, POINTER(vp)]),
            "fhe_mul_relin": (ci, [vp, vp, vp, vp, POINTER(vp)]),
            "fhe_compare_lt": (ci, [vp, vp, vp, vp, ci, POINTER(vp)]),
            "fhe_compare_eq": (ci, [vp, vp, vp, vp, ci, POINTER(vp)]),
            "fhe_compare": (ci, [vp, vp, vp, vp, ci, POINTER(vp), POINTER(vp)]),
            "fhe_max_min": (ci, [vp, vp, vp, vp, ci, vp, vp]),
            "fhe_max": (ci, [vp, vp, vp, vp, ci, vp]),
            "fhe_min": (ci, [vp, vp, vp, vp, ci, vp]),
            "fhe_trace_enable": (ci, [vp, ci]),
            "fhe_trace_get": (ci, [vp, vp, vp, ci]),
            "fhe_ntt_forward": (ci, [vp, vp, vp, ci]),
            "fhe_ntt_forward_batch": (ci, [vp, vp, ci, ci]),
            "fhe_ntt_inverse_batch": (ci, [vp, vp, ci, ci]),
            "fhe_ntt_inverse": (ci, [vp, vp, vp, ci]),
            "fhe_selftest_modarith": (ci, [u64, u64, u64, ci, ci]),
            "fhe_ctx_profile": (ci, [vp, ci]),
            "fhe_ctx_autotune": (ci, [vp, ci]),
            "fhe_ctx_ntt_variant": (ci, [vp, ci, vp]),
            "fhe_batch_submit": (ci, [vp, ci, POINTER(vp)]),
            "fhe_batch_submit_ex": (ci, [vp, ci, ci, POINTER(vp)]),
            "fhe_batch_wait": (ci, [vp, ci]),
            "fhe_batch_job_done": (ci, [vp, ci]),
            "fhe_batch_destroy": (None, [vp]),
            "fhe_job_footprint": (ctypes.c_uint64, [vp]),
            "fhe_ctx_inject_alloc_failure": (ci, [vp, ctypes.c_int64]),
            "fhe_ctx_trim": (ci, [vp]),
            "fhe_add_plain": (ci, [vp, vp, vp, POINTER(vp)]),
            "fhe_sub_plain": (ci, [vp, vp, vp, POINTER(vp)]),
            "fhe_mul_plain": (ci, [vp, vp, vp, POINTER(vp)]),
            "fhe_sort_galois": (ci, [vp, vp, ci]),
            "fhe_probe_bfly_peak": (ci, [vp]),
            "fhe_ct_serialize": (ci, [vp, vp, vp, u64, POINTER(c_uint64)]),
            "fhe_ct_deserialize": (ci, [vp, vp, u64, POINTER(vp)]),
            "fhe_server_cancel": (ci, [vp, c_uint64]),
            "fhe_sort_joint": (ci, [vp, vp, vp, ci, ci, POINTER(vp)]),
            "fhe_sort_ranks": (ci, [vp, vp, vp, ci, ci, POINTER(vp), vp]),
            "fhe_private_query": (ci, [vp, vp, vp, vp, vp, ci, vp, ci, POINTER(vp)]),
            "fhe_private_query_plan": (ci, [vp, vp, vp, vp, vp, ci, vp, ci, POINTER(vp)]),
            "fhe_ext_galois": (ci, [vp, ci, vp, ci]),
            "fhe_encrypt_ext": (ci, [vp, vp, vp, ci, ci, u64, POINTER(vp)]),
            "fhe_encrypt_ext_explicit": (ci, [vp, vp, vp, ci, ci, vp, vp, vp, POINTER(vp)]),
            "fhe_decrypt_ext": (ci, [vp, vp, vp, ci, vp]),
            "fhe_extract_digits": (ci, [vp, vp, vp, ci, POINTER(vp)]),
            "fhe_slot_plan": (ci, [ci, i64, ci, vp, vp, vp, ci, vp]),
            "fhe_slot_pack": (ci, [vp, vp, vp, ci, vp, POINTER(vp), ci]),
            "fhe_sort": (ci, [vp, vp, vp, ci, vp]),
            "fhe_compare_bivariate": (ci, [vp, vp, vp, vp, ci, POINTER(vp), POINTER(vp)]),
            "fhe_probe_int_peak": (ci, [POINTER(ctypes.c_double), POINTER(ctypes.c_double)]),
            "fhe_ctx_fused_modswitch": (ci, [vp, ci]),
            "fhe_ctx_set_batch_graphs": (ci, [vp, ci]),
            "fhe_ctx_memory_peak": (ci, [vp, POINTER(ctypes.c_uint64), ci]),
            "fhe_server_start": (ci, [vp, POINTER(vp)]),
            "fhe_server_submit": (ci, [vp, vp, POINTER(ctypes.c_uint64)]),
            "fhe_server_poll": (ci, [vp, ctypes.c_uint64, ci, vp]),
            "fhe_server_stats": (ci, [vp, vp]),
            "fhe_server_stop": (ci, [vp]),
            "fhe_tournament_galois": (ci, [vp, vp, ci]),
            "fhe_tournament": (ci, [vp, vp, vp, vp, vp, ci, u64, vp, vp]),
            "fhe_refresh_explicit": (ci, [vp, vp, vp, vp, vp, vp, vp, POINTER(vp)]),
            "fhe_refresh": (ci, [vp, vp, vp, vp, u64, POINTER(vp)]),
            "fhe_philox_blocks": (ci, [u64, ctypes.c_uint32, ci, vp]),
            "fhe_compare_plan": (ci, [vp, vp, vp, vp, ci, ci, ci, ci, POINTER(vp)]),
            "fhe_plan_run": (ci, [vp]),
            "fhe_plan_result": (ci, [vp, ci, POINTER(vp)]),
            "fhe_plan_nodes": (ci, [vp]),
            "fhe_plan_destroy": (None, [vp]),
            "fhe_mod_switch_noalloc": (ci, [vp, vp, vp, ci, ci, ci]),
            "fhe_ctx_profile_read": (ci, [vp, vp, vp, vp, vp, ci]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(c_void_p)


def _check(rc, ctx=None):
    if rc < 0:
        msg = lib().fhe_last_error(ctx).decode() if ctx else ""
        raise FheError(rc, msg)
    return rc


# ---------------------------------------------------------------------------
# device memory from PyTorch
# ---------------------------------------------------------------------------

def torch_allocator(device: int = 0):
    """An fhe_allocator whose calls go to torch's CUDA caching allocator."""
    import torch

    def _a(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
        except Exception:  # noqa: BLE001 -- reported to the library as NULL
            return None

    def _f(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = fhe_allocator(ALLOC_FN(_a), FREE_FN(_f), None)
    a._keep = (_a, _f)  # keep the Python callables alive
    return a


# ---------------------------------------------------------------------------
# wrappers with the C names
# ---------------------------------------------------------------------------

# allocator callbacks of live contexts: the library calls them until
# fhe_ctx_destroy, so they must not be garbage-collected before
_ALLOCATORS = {}


def fhe_ctx_create(log_n, p, L, K, prime_mod, prime_lo, prime_hi, allocator=None, stream=None):
    P = fhe_params(log_n, p, L, K, prime_mod, prime_lo, prime_hi)
    out = c_void_p()
    rc = lib().fhe_ctx_create(ctypes.byref(P), ctypes.byref(allocator) if allocator is not None else None,
                              c_void_p(stream or 0), ctypes.byref(out))
    _check(rc)
    if allocator is not None:
        _ALLOCATORS[out.value] = allocator
    return out


def fhe_ctx_destroy(ctx):
    lib().fhe_ctx_destroy(ctx)
    _ALLOCATORS.pop(ctx.value if isinstance(ctx, c_void_p) else ctx, None)


def fhe_ctx_info(ctx) -> fhe_info:
    i = fhe_info()
    _check(lib().fhe_ctx_info(ctx, ctypes.byref(i)), ctx)
    return i


def fhe_ctx_primes(ctx):
    info = fhe_ctx_info(ctx)
    out = np.zeros(info.L + info.K, dtype=np.uint64)
    _check(lib().fhe_ctx_primes(ctx, _ptr(out)), ctx)
    return [int(x) for x in out]


def fhe_ctx_sync(ctx):
    _check(lib().fhe_ctx_sync(ctx), ctx)


def fhe_ctx_set_stream(ctx, stream: int):
    _check(lib().fhe_ctx_set_stream(ctx, c_void_p(stream)), ctx)


def fhe_ctx_memory(ctx):
    r, u = c_uint64(), c_uint64()
    _check(lib().fhe_ctx_memory(ctx, ctypes.byref(r), ctypes.byref(u)), ctx)
    return r.value, u.value


def fhe_ctx_set_budget(ctx, nbytes: int):
    _check(lib().fhe_ctx_set_budget(ctx, nbytes), ctx)


def fhe_ctx_launches(ctx) -> int:
    return int(lib().fhe_ctx_launches(ctx))


def fhe_keygen_explicit(ctx, s, a, e):
    s = np.ascontiguousarray(s, dtype=np.int64)
    a = np.ascontiguousarray(a, dtype=np.uint64)
    e = np.ascontiguousarray(e, dtype=np.int64)
    sk, pk = c_void_p(), c_void_p()
    _check(lib().fhe_keygen_explicit(ctx, _ptr(s), _ptr(a), _ptr(e), ctypes.byref(sk), ctypes.byref(pk)), ctx)
    return sk, pk


def fhe_keygen(ctx, seed: int):
    sk, pk = c_void_p(), c_void_p()
    _check(lib().fhe_keygen(ctx, seed, ctypes.byref(sk), ctypes.byref(pk)), ctx)
    return sk, pk


def fhe_sk_destroy(sk):
    lib().fhe_sk_destroy(sk)


def fhe_pk_destroy(pk):
    lib().fhe_pk_destroy(pk)


def fhe_evk_create_explicit(ctx, sk, galois, a, e):
    g = np.ascontiguousarray(galois, dtype=np.int64) if len(galois) else np.zeros(1, dtype=np.int64)
    a = np.ascontiguousarray(a, dtype=np.uint64)
    e = np.ascontiguousarray(e, dtype=np.int64)
    out = c_void_p()
    _check(lib().fhe_evk_create_explicit(ctx, sk, _ptr(g), len(galois), _ptr(a), _ptr(e), ctypes.byref(out)), ctx)
    return out


def fhe_evk_create(ctx, sk, galois, seed: int):
    g = np.ascontiguousarray(galois, dtype=np.int64) if len(galois) else np.zeros(1, dtype=np.int64)
    out = c_void_p()
    _check(lib().fhe_evk_create(ctx, sk, _ptr(g), len(galois), seed, ctypes.byref(out)), ctx)
    return out


def fhe_evk_destroy(evk):
    lib().fhe_evk_destroy(evk)


def fhe_encrypt_explicit(ctx, pk, slots, u, e0, e1):
    slots = np.ascontiguousarray(slots, dtype=np.uint64)
    count = slots.shape[0]
    u = np.ascontiguousarray(u, dtype=np.int64)
    e0 = np.ascontiguousarray(e0, dtype=np.int64)
    e1 = np.ascontiguousarray(e1, dtype=np.int64)
    out = c_void_p()
    _check(lib().fhe_encrypt_explicit(ctx, pk, _ptr(slots), count, _ptr(u), _ptr(e0), _ptr(e1), ctypes.byref(out)),
           ctx)
    return out


def fhe_encrypt(ctx, pk, slots, seed: int):
    slots = np.ascontiguousarray(slots, dtype=np.uint64)
    out = c_void_p()
    _check(lib().fhe_encrypt(ctx, pk, _ptr(slots), slots.shape[0], seed, ctypes.byref(out)), ctx)
    return out


def fhe_ct_shape(ct):
    c, n, l = c_int(), c_int(), c_int()
    _check(lib().fhe_ct_shape(ct, ctypes.byref(c), ctypes.byref(n), ctypes.byref(l)))
    return c.value, n.value, l.value


def fhe_decrypt(ctx, sk, ct):
    count, _, _ = fhe_ct_shape(ct)
    info = fhe_ctx_info(ctx)
    out = np.zeros((count, info.slots), dtype=np.uint64)
    _check(lib().fhe_decrypt(ctx, sk, ct, _ptr(out)), ctx)
    return out


def fhe_refresh_explicit(ctx, sk, pk, ct, u, e0, e1):
    u = np.ascontiguousarray(u, dtype=np.int64)
    e0 = np.ascontiguousarray(e0, dtype=np.int64)
    e1 = np.ascontiguousarray(e1, dtype=np.int64)
    out = c_void_p()
    _check(lib().fhe_refresh_explicit(ctx, sk, pk, ct, _ptr(u), _ptr(e0), _ptr(e1), ctypes.byref(out)), ctx)
    return out


def fhe_refresh(ctx, sk, pk, ct, seed: int):
    out = c_void_p()
    _check(lib().fhe_refresh(ctx, sk, pk, ct, seed, ctypes.byref(out)), ctx)
    return out


def fhe_philox_blocks(seed: int, tag: int, n: int):
    out = np.zeros(4 * n, dtype=np.uint32)
    _check(lib().fhe_philox_blocks(seed, tag, n, _ptr(out)))
    return out.reshape(n, 4)


def fhe_ct_destroy(ct):
    lib().fhe_ct_destroy(ct)


def fhe_ct_serialize(ctx, ct) -> bytes:
    """The ciphertext batch as a checkpoint image (header, primes, limbs)."""
    n = c_uint64()
    _check(lib().fhe_ct_serialize(ctx, ct, None, 0, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().fhe_ct_serialize(ctx, ct, buf, n.value, ctypes.byref(n)), ctx)
    return buf.raw


def fhe_ct_deserialize(ctx, image: bytes):
    out = c_void_p()
    _check(lib().fhe_ct_deserialize(ctx, image, len(image), ctypes.byref(out)), ctx)
    return out


def fhe_ct_export_coeff(ctx, ct):
    count, npoly, level = fhe_ct_shape(ct)
    N = fhe_ctx_info(ctx).N
    out = np.zeros((count, npoly, level, N), dtype=np.uint64)
    _check(lib().fhe_ct_export_coeff(ctx, ct, _ptr(out)), ctx)
    return out


def fhe_ct_import_coeff(ctx, data):
    data = np.ascontiguousarray(data, dtype=np.uint64)
    count, npoly, level, _ = data.shape
    out = c_void_p()
    _check(lib().fhe_ct_import_coeff(ctx, _ptr(data), count, npoly, level, ctypes.byref(out)), ctx)
    return out


def fhe_ct_load_coeff(ctx, ct, data):
    data = np.ascontiguousarray(data, dtype=np.uint64)
    _check(lib().fhe_ct_load_coeff(ctx, ct, _ptr(data)), ctx)


def _binary(name):
    def f(ctx, a, b):
        out = c_void_p()
        _check(getattr(lib(), name)(ctx, a, b, ctypes.byref(out)), ctx)
        return out

    f.__name__ = name
    return f


fhe_add = _binary("fhe_add")
fhe_sub = _binary("fhe_sub")
fhe_mul = _binary("fhe_mul")


def fhe_neg(ctx, a):
    out = c_void_p()
    _check(lib().fhe_neg(ctx, a, ctypes.byref(out)), ctx)
    return out


def fhe_mul_const(ctx, a, k: int):
    out = c_void_p()
    _check(lib().fhe_mul_const(ctx, a, int(k), ctypes.byref(out)), ctx)
    return out


def fhe_add_const(ctx, a, k: int):
    out = c_void_p()
    _check(lib().fhe_add_const(ctx, a, int(k), ctypes.byref(out)), ctx)
    return out


def fhe_relinearize(ctx, evk, a):
    out = c_void_p()
    _check(lib().fhe_relinearize(ctx, evk, a, ctypes.byref(out)), ctx)
    return out


def fhe_mod_switch(ctx, a, level: int):
    out = c_void_p()
    _check(lib().fhe_mod_switch(ctx, a, level, ctypes.byref(out)), ctx)
    return out


def fhe_rotate(ctx, evk, a, galois: int):
    out = c_void_p()
    _check(lib().fhe_rotate(ctx, evk, a, int(galois), ctypes.byref(out)), ctx)
    return out


def fhe_mul_relin(ctx, evk, a, b):
    out = c_void_p()
    _check(lib().fhe_mul_relin(ctx, evk, a, b, ctypes.byref(out)), ctx)
    return out


def _handles(cts):
    arr = (c_void_p * len(cts))(*[c.value if isinstance(c, c_void_p) else c for c in cts])
    return arr


def fhe_compare(ctx, evk, xs, ys, want_lt=True, want_eq=True):
    lt, eq = c_void_p(), c_void_p()
    _check(lib().fhe_compare(ctx, evk, _handles(xs), _handles(ys), len(xs),
                             ctypes.byref(lt) if want_lt else None, ctypes.byref(eq) if want_eq else None), ctx)
    return (lt if want_lt else None), (eq if want_eq else None)


def fhe_compare_lt(ctx, evk, xs, ys):
    out = c_void_p()
    _check(lib().fhe_compare_lt(ctx, evk, _handles(xs), _handles(ys), len(xs), ctypes.byref(out)), ctx)
    return out


def fhe_compare_eq(ctx, evk, xs, ys):
    out = c_void_p()
    _check(lib().fhe_compare_eq(ctx, evk, _handles(xs), _handles(ys), len(xs), ctypes.byref(out)), ctx)
    return out


def fhe_compare_bivariate(ctx, evk, xs, ys, want_lt=True, want_eq=True):
    """LT / EQ of full digits in [0, p) by the bivariate circuit."""
    lt, eq = c_void_p(), c_void_p()
    _check(lib().fhe_compare_bivariate(ctx, evk, _handles(xs), _handles(ys), len(xs),
                                       ctypes.byref(lt) if want_lt else None, ctypes.byref(eq) if want_eq else None),
           ctx)
    return (lt if want_lt else None), (eq if want_eq else None)


def _plain_op(name):
    def f(ctx, a, slots):
        v = np.ascontiguousarray(slots, dtype=np.uint64)
        out = c_void_p()
        _check(getattr(lib(), name)(ctx, a, _ptr(v), ctypes.byref(out)), ctx)
        return out

    f.__name__ = name
    return f


fhe_add_plain = _plain_op("fhe_add_plain")
fhe_sub_plain = _plain_op("fhe_sub_plain")
fhe_mul_plain = _plain_op("fhe_mul_plain")


def fhe_sort_galois(ctx):
    n = _check(lib().fhe_sort_galois(ctx, None, 0), ctx)
    g = np.zeros(max(n, 1), dtype=np.int64)
    lib().fhe_sort_galois(ctx, _ptr(g), n)
    return [int(v) for v in g[:n]]


FHE_QUERY_OVERLAP = 1


def fhe_private_query(ctx, evk, q, data, op1, op2: int, codes, overlap: bool = True):
    """sum over the three candidates (data + op1, data * op1, data^op2) of
    candidate * EQ(q, code); overlap runs the comparison branch concurrently
    with the arithmetic."""
    cd = np.ascontiguousarray(np.asarray(codes, dtype=np.int64))
    assert cd.shape == (3,)
    out = c_void_p()
    _check(lib().fhe_private_query(ctx, evk, q, data, op1, int(op2), _ptr(cd),
                                   FHE_QUERY_OVERLAP if overlap else 0, ctypes.byref(out)), ctx)
    return out


def fhe_private_query_plan(ctx, evk, q, data, op1, op2: int, codes, serial: bool = False):
    """The private query captured as a graph; fhe_plan_run replays it and
    fhe_plan_result(plan, 0) is the answer."""
    cd = np.ascontiguousarray(np.asarray(codes, dtype=np.int64))
    assert cd.shape == (3,)
    out = c_void_p()
    _check(lib().fhe_private_query_plan(ctx, evk, q, data, op1, int(op2), _ptr(cd),
                                        FHE_PLAN_SERIAL if serial else 0, ctypes.byref(out)), ctx)
    return out


def fhe_ext_galois(ctx, d: int):
    n = _check(lib().fhe_ext_galois(ctx, int(d), None, 0), ctx)
    g = np.zeros(max(n, 1), dtype=np.int64)
    lib().fhe_ext_galois(ctx, int(d), _ptr(g), n)
    return [int(v) for v in g[:n]]


def _ext_digits(ctx, digits, d):
    ns = fhe_ctx_info(ctx).slots
    a = np.ascontiguousarray(np.asarray(digits, dtype=np.uint64))
    if a.ndim == 2:
        a = a[None]
    if a.ndim != 3 or a.shape[1:] != (ns, d):
        raise ValueError(f"digits must be (count, {ns}, {d})")
    return a


def fhe_encrypt_ext(ctx, pk, digits, d: int, seed: int):
    """digits (count, n_s, d) in [0, p): each slot the F_{p^d} element
    sum_k digits[.., k] Y'^k."""
    a = _ext_digits(ctx, digits, d)
    out = c_void_p()
    _check(lib().fhe_encrypt_ext(ctx, pk, _ptr(a), a.shape[0], int(d), seed, ctypes.byref(out)), ctx)
    return out


def fhe_encrypt_ext_explicit(ctx, pk, digits, d: int, u, e0, e1):
    a = _ext_digits(ctx, digits, d)
    u, e0, e1 = (np.ascontiguousarray(x, dtype=np.int64) for x in (u, e0, e1))
    out = c_void_p()
    _check(lib().fhe_encrypt_ext_explicit(ctx, pk, _ptr(a), a.shape[0], int(d), _ptr(u), _ptr(e0), _ptr(e1),
                                          ctypes.byref(out)), ctx)
    return out


def fhe_decrypt_ext(ctx, sk, ct, d: int):
    count = fhe_ct_shape(ct)[0]
    ns = fhe_ctx_info(ctx).slots
    out = np.zeros((count, ns, d), dtype=np.uint64)
    _check(lib().fhe_decrypt_ext(ctx, sk, ct, int(d), _ptr(out)), ctx)
    return out


def fhe_extract_digits(ctx, evk, ct, d: int):
    """The d digit ciphertexts (F_p constants) of an F_{p^d}-slot ciphertext."""
    out = (c_void_p * d)()
    _check(lib().fhe_extract_digits(ctx, evk, ct, int(d), out), ctx)
    return [c_void_p(out[k]) for k in range(d)]


def _useful(ns, useful):
    u = np.ascontiguousarray(np.asarray(useful, dtype=bool).astype(np.uint8))
    if u.ndim != 2 or u.shape[1] != ns:
        raise ValueError(f"useful must be (inputs, {ns})")
    return u


def fhe_slot_plan(slots: int, ring_n: int, useful):
    """Host-only placement: (number of outputs, dest (inputs x n_s: output *
    n_s + slot or -1), rotation elements the plan needs)."""
    u = _useful(slots, useful)
    n = u.shape[0]
    dest = np.zeros(u.shape, dtype=np.int32)
    ng = ctypes.c_int(0)
    _check(lib().fhe_slot_plan(int(slots), int(ring_n), n, _ptr(u), _ptr(dest), None, 0, ctypes.byref(ng)))
    g = np.zeros(max(ng.value, 1), dtype=np.int64)
    n_out = _check(lib().fhe_slot_plan(int(slots), int(ring_n), n, _ptr(u), None, _ptr(g), ng.value, None))
    return n_out, dest, [int(v) for v in g[:ng.value]]


def fhe_slot_pack(ctx, evk, cts, useful):
    """The inputs' useful slots compacted into as few ciphertexts as the plan
    needs (handles, caller-owned)."""
    u = _useful(fhe_ctx_info(ctx).slots, useful)
    if u.shape[0] != len(cts):
        raise ValueError("one row of useful per input")
    out = (c_void_p * max(len(cts), 1))()
    n = _check(lib().fhe_slot_pack(ctx, evk, _handles(cts), len(cts), _ptr(u), out, len(cts)), ctx)
    return [c_void_p(out[i]) for i in range(n)]


def fhe_sort(ctx, evk, xs):
    """Every row of every ciphertext sorted; xs: the d digit handles."""
    d = len(xs)
    out = (c_void_p * d)()
    _check(lib().fhe_sort(ctx, evk, _handles(xs), d, out), ctx)
    return [c_void_p(v) for v in out]


def fhe_sort_joint(ctx, evk, cts):
    """Row r of the K batches cts[a] (each a list of d digit handles) sorted as
    one sequence; returns K lists of d handles (batch t: positions t cols ..)."""
    K, d = len(cts), len(cts[0])
    out = (c_void_p * (K * d))()
    _check(lib().fhe_sort_joint(ctx, evk, _handles([h for xs in cts for h in xs]), K, d, out), ctx)
    return [[c_void_p(out[t * d + k]) for k in range(d)] for t in range(K)]


def fhe_sort_ranks(ctx, evk, cts, matrix=False):
    """Ranks (mod p) of every value of row r of the K batches cts[a] (lists of
    d digit handles), any K cols; with matrix=True also the comparison matrix
    as a dict (a, b, s) -> handle.  Returns (ranks, matrix or None)."""
    K, d = len(cts), len(cts[0])
    cols = fhe_ctx_info(ctx).slots // 2
    ranks = (c_void_p * K)()
    mat = (c_void_p * (K * K * cols))() if matrix else None
    _check(lib().fhe_sort_ranks(ctx, evk, _handles([h for xs in cts for h in xs]), K, d, ranks,
                                ctypes.cast(mat, c_void_p) if mat is not None else None), ctx)
    m = None
    if matrix:
        m = {(a, b, s): c_void_p(mat[(a * K + b) * cols + s]) for a in range(K) for b in range(K) for s in range(cols)
             if not (a == b and s == 0)}
    return [c_void_p(ranks[a]) for a in range(K)], m


def fhe_max_min(ctx, evk, xs, ys):
    d = len(xs)
    mx, mn = (c_void_p * d)(), (c_void_p * d)()
    _check(lib().fhe_max_min(ctx, evk, _handles(xs), _handles(ys), d, mx, mn), ctx)
    return [c_void_p(v) for v in mx], [c_void_p(v) for v in mn]


FHE_PLAN_SERIAL = 1
FHE_PLAN_BIVARIATE = 2


def fhe_compare_plan(ctx, evk, xs, ys, want_lt=True, want_eq=True, flags=0):
    out = c_void_p()
    _check(lib().fhe_compare_plan(ctx, evk, _handles(xs), _handles(ys), len(xs), int(want_lt), int(want_eq),
                                  int(flags), ctypes.byref(out)), ctx)
    return out


def fhe_plan_run(plan, ctx=None):
    _check(lib().fhe_plan_run(plan), ctx)


def fhe_plan_result(plan, which: int):
    out = c_void_p()
    _check(lib().fhe_plan_result(plan, which, ctypes.byref(out)))
    return out


def fhe_plan_nodes(plan) -> int:
    return int(lib().fhe_plan_nodes(plan))


def fhe_plan_destroy(plan):
    lib().fhe_plan_destroy(plan)


def fhe_tournament_galois(ctx):
    n = _check(lib().fhe_tournament_galois(ctx, None, 0), ctx)
    out = np.zeros(max(n, 1), dtype=np.int64)
    lib().fhe_tournament_galois(ctx, _ptr(out), n)
    return [int(v) for v in out[:n]]


def fhe_tournament(ctx, evk, sk, pk, xs, seed: int, want_max=True, want_min=True):
    d = len(xs)
    mx, mn = (c_void_p * d)(), (c_void_p * d)()
    _check(lib().fhe_tournament(ctx, evk, sk, pk, _handles(xs), d, seed, mx if want_max else None,
                                mn if want_min else None), ctx)
    return ([c_void_p(v) for v in mx] if want_max else None), ([c_void_p(v) for v in mn] if want_min else None)


class Job:
    """A request for fhe_batch_submit; after the batch completes, .out0 and
    .out1 hold the result handles (LT / EQ, or the max / min digits)."""

    def __init__(self, ctx, evk, kind, xs, ys, want0=True, want1=True):
        self.ctx, self.evk, self.kind, self.d = ctx, evk, kind, len(xs)
        self._x = _handles(xs)
        self._y = _handles(ys) if ys is not None else None
        n = self.d if kind in (FHE_JOB_MAXMIN, FHE_JOB_SORT) else 1
        self._o0 = (c_void_p * n)() if want0 else None
        self._o1 = (c_void_p * n)() if want1 and kind != FHE_JOB_SORT else None

    def struct(self):
        return fhe_job(self.ctx.value if isinstance(self.ctx, c_void_p) else self.ctx,
                       self.evk.value if isinstance(self.evk, c_void_p) else self.evk, self.kind, self.d,
                       ctypes.cast(self._x, c_void_p),
                       ctypes.cast(self._y, c_void_p) if self._y is not None else None,
                       ctypes.cast(self._o0, c_void_p) if self._o0 is not None else None,
                       ctypes.cast(self._o1, c_void_p) if self._o1 is not None else None)

    @property
    def out0(self):
        return None if self._o0 is None else [c_void_p(v) for v in self._o0]

    @property
    def out1(self):
        return None if self._o1 is None else [c_void_p(v) for v in self._o1]


FHE_BATCH_ALIGN_LEVELS = 1
FHE_BATCH_FUSE_RINGS = 2


def fhe_batch_submit(jobs, flags: int = 0):
    arr = (fhe_job * len(jobs))(*[j.struct() for j in jobs])
    out = c_void_p()
    _check(lib().fhe_batch_submit_ex(ctypes.cast(arr, c_void_p), len(jobs), int(flags), ctypes.byref(out)),
           jobs[0].ctx if jobs else None)
    return out


def fhe_batch_wait(batch, timeout_ms: int) -> int:
    """0 when complete, FHE_ETIMEOUT (-6) if still running after timeout_ms."""
    rc = lib().fhe_batch_wait(batch, int(timeout_ms))
    if rc < 0 and rc != -6:
        _check(rc)
    return rc


def fhe_batch_job_done(batch, i: int) -> bool:
    """True once job i of the batch has its results (no waiting)."""
    return _check(lib().fhe_batch_job_done(batch, int(i))) == 1


def fhe_batch_destroy(batch):
    lib().fhe_batch_destroy(batch)


def fhe_ctx_set_batch_graphs(ctx, max_plans: int):
    _check(lib().fhe_ctx_set_batch_graphs(ctx, int(max_plans)), ctx)


def fhe_ctx_fused_modswitch(ctx, on: bool):
    _check(lib().fhe_ctx_fused_modswitch(ctx, int(bool(on))), ctx)


def fhe_probe_bfly_peak():
    v = ctypes.c_double()
    _check(lib().fhe_probe_bfly_peak(ctypes.byref(v)))
    return v.value


def fhe_probe_int_peak():
    """(32-bit multiply-adds/s, 64-bit high products/s) measured on the current device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().fhe_probe_int_peak(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def fhe_ctx_trim(ctx):
    _check(lib().fhe_ctx_trim(ctx), ctx)


def fhe_ctx_inject_alloc_failure(ctx, n: int):
    _check(lib().fhe_ctx_inject_alloc_failure(ctx, int(n)), ctx)


def fhe_ctx_memory_peak(ctx, reset: bool = False) -> int:
    v = ctypes.c_uint64()
    _check(lib().fhe_ctx_memory_peak(ctx, ctypes.byref(v), int(reset)), ctx)
    return v.value


def fhe_job_footprint(job: "Job") -> int:
    st = job.struct()
    return int(lib().fhe_job_footprint(ctypes.byref(st)))


def fhe_server_start(hbm_budget: int = 0, max_batch: int = 0, batch_flags: int = 0):
    cfg = fhe_server_config(int(hbm_budget), int(max_batch), int(batch_flags))
    out = c_void_p()
    _check(lib().fhe_server_start(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def fhe_server_submit(server, job: "Job") -> int:
    """Queues the job; the Job object must stay alive (its output arrays
    receive the handles) until fhe_server_poll reports it done."""
    st = job.struct()
    t = ctypes.c_uint64()
    _check(lib().fhe_server_submit(server, ctypes.byref(st), ctypes.byref(t)), job.ctx)
    return t.value


def fhe_server_poll(server, ticket: int, timeout_ms: int = 0):
    """(done, fhe_request_info)."""
    info = fhe_request_info()
    rc = _check(lib().fhe_server_poll(server, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(info)))
    return rc == 1, info


def fhe_server_cancel(server, ticket: int) -> int:
    """0 if the queued request was canceled; FHE_EBUSY (-11) if it already
    runs or is done."""
    rc = lib().fhe_server_cancel(server, ctypes.c_uint64(ticket))
    if rc < 0 and rc != -11:
        _check(rc)
    return rc


def fhe_server_stats(server) -> fhe_server_status:
    st = fhe_server_status()
    _check(lib().fhe_server_stats(server, ctypes.byref(st)))
    return st


def fhe_server_stop(server):
    _check(lib().fhe_server_stop(server))


def fhe_ctx_autotune(ctx, njobs: int) -> int:
    return _check(lib().fhe_ctx_autotune(ctx, njobs), ctx)


def fhe_ctx_ntt_variant(ctx, set_variant: int = -1):
    """(chosen variant, [ms of variants 0, 1, 2, 3]; 0 where a variant does not exist)."""
    ms = np.zeros(4, dtype=np.float32)
    v = _check(lib().fhe_ctx_ntt_variant(ctx, set_variant, _ptr(ms)), ctx)
    return v, [float(x) for x in ms]


def fhe_trace_enable(ctx, on: bool):
    _check(lib().fhe_trace_enable(ctx, 1 if on else 0), ctx)


def fhe_trace_get(ctx):
    n = _check(lib().fhe_trace_get(ctx, None, None, 0), ctx)
    ops = np.zeros(max(n, 1), dtype=np.int32)
    lv = np.zeros(max(n, 1), dtype=np.int32)
    lib().fhe_trace_get(ctx, _ptr(ops), _ptr(lv), n)
    return [(OPS[int(o)], int(v)) for o, v in zip(ops[:n], lv[:n])]


def fhe_ntt_forward(ctx, dev_ptr: int, prime_idx, nlimbs: int):
    pi = np.ascontiguousarray(prime_idx, dtype=np.int32)
    _check(lib().fhe_ntt_forward(ctx, c_void_p(dev_ptr), _ptr(pi), nlimbs), ctx)


def fhe_ntt_forward_batch(ctx, dev_ptr: int, count: int, nprimes: int):
    _check(lib().fhe_ntt_forward_batch(ctx, c_void_p(dev_ptr), count, nprimes), ctx)


def fhe_ntt_inverse_batch(ctx, dev_ptr: int, count: int, nprimes: int):
    _check(lib().fhe_ntt_inverse_batch(ctx, c_void_p(dev_ptr), count, nprimes), ctx)


def fhe_ntt_inverse(ctx, dev_ptr: int, prime_idx, nlimbs: int):
    pi = np.ascontiguousarray(prime_idx, dtype=np.int32)
    _check(lib().fhe_ntt_inverse(ctx, c_void_p(dev_ptr), _ptr(pi), nlimbs), ctx)


def fhe_mod_switch_noalloc(ctx, in_ptr: int, out_ptr: int, count: int, npoly: int, level: int):
    """Modulus switch of caller-owned device buffers (raw device addresses),
    for callers that cannot allocate device memory; see include/fhe.h."""
    _check(lib().fhe_mod_switch_noalloc(ctx, c_void_p(in_ptr), c_void_p(out_ptr), count, npoly, level), ctx)


KERNEL_CLASSES = ["ntt_fwd", "ntt_inv", "ntt_modup", "ntt_moddown", "ntt_modswitch", "ks_inner", "tensor",
                  "elementwise", "automorphism"]


def fhe_ctx_profile(ctx, on: bool):
    _check(lib().fhe_ctx_profile(ctx, 1 if on else 0), ctx)


def fhe_ctx_profile_read(ctx):
    """{class: (ms, launches, algorithmic bytes, butterflies)} since the last read."""
    n = len(KERNEL_CLASSES)
    ms = np.zeros(n, dtype=np.float64)
    cnt = np.zeros(n, dtype=np.int64)
    by = np.zeros(n, dtype=np.float64)
    bf = np.zeros(n, dtype=np.float64)
    _check(lib().fhe_ctx_profile_read(ctx, _ptr(ms), _ptr(cnt), _ptr(by), _ptr(bf), n), ctx)
    return {k: (float(ms[i]), int(cnt[i]), float(by[i]), float(bf[i])) for i, k in enumerate(KERNEL_CLASSES)}


def fhe_selftest_modarith(prime_mod, prime_lo, prime_hi, nprimes, iters) -> int:
    return int(lib().fhe_selftest_modarith(prime_mod, prime_lo, prime_hi, nprimes, iters))
