"""Builds library contexts, keys and ciphertexts from the same seeded inputs as
tests/oracle_setup.py, so both sides see identical randomness."""
from __future__ import annotations

import numpy as np

from paper_2407_07308_gb300 import fhe, synth


class GpuSetup:
    def __init__(self, logN, p, L, K, U, lo, hi, seed=1, galois=(), d=1, use_torch_alloc=True):
        import torch

        self.torch = torch
        self.alloc = fhe.torch_allocator(0) if use_torch_alloc else None
        self.ctx = fhe.fhe_ctx_create(logN, p, L, K, U, lo, hi, allocator=self.alloc)
        self.info = fhe.fhe_ctx_info(self.ctx)
        self.N, self.p, self.L, self.K = self.info.N, p, L, K
        self.ns = self.info.slots
        self.primes = fhe.fhe_ctx_primes(self.ctx)
        self.galois = list(galois)
        km = synth.KeyMaterial(seed, self.primes, L, K, self.N, n_galois=len(self.galois))
        self.km = km
        self.sk, self.pk = fhe.fhe_keygen_explicit(self.ctx, km.s, km.a_pk, km.e_pk)
        self.evk = fhe.fhe_evk_create_explicit(self.ctx, self.sk, self.galois, km.a_ksk, km.e_ksk)
        self._owned = []

    def encrypt_slots(self, slot_rows, seed):
        """One batch handle holding one ciphertext per row (same randomness
        order as OracleSetup.encrypt_slots)."""
        rows = np.asarray(slot_rows, dtype=np.uint64).reshape(-1, self.ns)
        r = synth.EncRandomness(seed, rows.shape[0], self.N)
        return self.own(fhe.fhe_encrypt_explicit(self.ctx, self.pk, rows, r.u, r.e0, r.e1))

    def encrypt_ext(self, digits, d, seed):
        """One batch handle of F_{p^d}-slot ciphertexts, digits (count, n_s,
        d) (same randomness order as OracleSetup.encrypt_coeffs)."""
        a = np.asarray(digits, dtype=np.uint64).reshape(-1, self.ns, d)
        r = synth.EncRandomness(seed, a.shape[0], self.N)
        return self.own(fhe.fhe_encrypt_ext_explicit(self.ctx, self.pk, a, d, r.u, r.e0, r.e1))

    def encrypt_each(self, slot_rows, seed):
        """One single-ciphertext handle per row."""
        rows = np.asarray(slot_rows, dtype=np.uint64).reshape(-1, self.ns)
        r = synth.EncRandomness(seed, rows.shape[0], self.N)
        return [self.own(fhe.fhe_encrypt_explicit(self.ctx, self.pk, rows[i:i + 1], r.u[i:i + 1], r.e0[i:i + 1],
                                                  r.e1[i:i + 1])) for i in range(rows.shape[0])]

    def own(self, h):
        self._owned.append(h)
        return h

    def decrypt(self, ct):
        return fhe.fhe_decrypt(self.ctx, self.sk, ct)

    def export(self, ct):
        return fhe.fhe_ct_export_coeff(self.ctx, ct)

    def close(self):
        for h in self._owned:
            fhe.fhe_ct_destroy(h)
        self._owned = []
        fhe.fhe_evk_destroy(self.evk)
        fhe.fhe_sk_destroy(self.sk)
        fhe.fhe_pk_destroy(self.pk)
        fhe.fhe_ctx_destroy(self.ctx)
        self.ctx = None
