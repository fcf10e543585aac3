"""Builds oracle contexts, keys and ciphertexts from the shared seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle.bgv import Oracle
from oracle.circuits import Evaluator
from oracle.encoding import SlotStructure
from paper_2407_07308_gb300 import synth


class OracleSetup:
    def __init__(self, logN, p, L, K, U, lo, hi, seed=1, galois=(), d=1):
        self.o = Oracle(logN, p, L, K, U, lo, hi)
        self.N, self.p, self.L, self.K = self.o.N, p, L, K
        self.ss = SlotStructure(p, self.N)
        self.galois = list(galois)
        self.km = synth.KeyMaterial(seed, self.o.primes, L, K, self.N, n_galois=len(self.galois))
        self.s = self.km.s
        self.pk = self.o.keygen(self.s, self.km.a_pk, self.km.e_pk)
        self.rlk = self.o.relin_key(self.s, self.km.a_ksk[0], self.km.e_ksk[0])
        self.gks = {g: self.o.galois_key(self.s, g, self.km.a_ksk[1 + i], self.km.e_ksk[1 + i])
                    for i, g in enumerate(self.galois)}

    def evaluator(self) -> Evaluator:
        return Evaluator(self.o, self.rlk, self.gks)

    def encrypt_slots(self, slot_rows, seed):
        """Encrypt each row of slot values (len n_s) into one ciphertext."""
        rows = np.asarray(slot_rows, dtype=np.int64).reshape(-1, self.ss.ns)
        r = synth.EncRandomness(seed, rows.shape[0], self.N)
        return [self.o.encrypt(self.pk, self.ss.encode(row), r.u[i], r.e0[i], r.e1[i])
                for i, row in enumerate(rows)]

    def decrypt_slots(self, ct):
        return self.ss.decode(self.o.decrypt_coeffs(ct, self.s))

    def encrypt_coeffs(self, coeff_rows, seed):
        """Encrypt each row of plaintext coefficients (len N) into one
        ciphertext, with the same randomness stream as encrypt_slots."""
        rows = np.asarray(coeff_rows, dtype=np.int64).reshape(-1, self.N)
        r = synth.EncRandomness(seed, rows.shape[0], self.N)
        return [self.o.encrypt(self.pk, row, r.u[i], r.e0[i], r.e1[i]) for i, row in enumerate(rows)]

    def encrypt_row(self, slot_rows, seed, idx):
        """Ciphertext idx of encrypt_slots(slot_rows, seed) alone (the same
        randomness rows), without encrypting the others."""
        rows = np.asarray(slot_rows, dtype=np.int64).reshape(-1, self.ss.ns)
        r = synth.EncRandomness(seed, rows.shape[0], self.N)
        return self.o.encrypt(self.pk, self.ss.encode(rows[idx]), r.u[idx], r.e0[idx], r.e1[idx])


def compare_one(job):
    """Worker (run in a spawned process): the oracle's LT and EQ limbs of
    ciphertext idx of a batch comparison whose digit k was encrypted from
    xd[k] / yd[k] with seeds xs[k] / ys[k].  Returns the (lt, eq)
    coefficient arrays and the comparison's operation trace."""
    params, seed, xd, yd, xs, ys, idx, level = job
    o = OracleSetup(seed=seed, **params)
    ev = o.evaluator()
    xo = [o.encrypt_row(xd[k], xs[k], idx) for k in range(len(xd))]
    yo = [o.encrypt_row(yd[k], ys[k], idx) for k in range(len(yd))]
    if level is not None:
        xo = [ev.lower(c, level) for c in xo]
        yo = [ev.lower(c, level) for c in yo]
    ev.trace.clear()
    lt, eq = ev.compare(xo, yo, True, True)
    return lt.data.copy(), eq.data.copy(), list(ev.trace)


def compare_many(jobs):
    """compare_one over several jobs in spawned processes (safe after the
    parent has initialised CUDA)."""
    import multiprocessing as mp

    if len(jobs) == 1:
        return [compare_one(jobs[0])]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        return pool.map(compare_one, jobs, chunksize=1)
