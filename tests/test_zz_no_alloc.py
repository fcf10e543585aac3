"""The allocation-free modulus switch (fhe_mod_switch_noalloc) against the
pool-based fhe_mod_switch.

fhe_mod_switch_noalloc serves callers that cannot allocate device memory (a
host framework that owns all of it, or a loop that must not pay for a
cudaMalloc): they pass their own input and output buffers and the library
uses a fixed scratch array.  This file is named to be collected last, so a
run that stops at the first failure has already run every other test."""
import random

import numpy as np
import pytest

from tests.params import CHAIN50

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCRATCH_WORDS = 1 << 20  # the library's fixed scratch (count * npoly * N at most)


def _to_device_ntt(fhe, g, coeff, npoly, level):
    """Caller-owned device copy of an exported ciphertext, NTT domain."""
    dev = torch.from_numpy(coeff.view(np.int64).copy()).cuda()
    limbs = coeff.shape[0] * npoly * level
    fhe.fhe_ntt_forward(g.ctx, dev.data_ptr(), [i % level for i in range(limbs)], limbs)
    return dev


def _from_device_ntt(fhe, g, dev, npoly, level):
    limbs = dev.shape[0] * npoly * level
    fhe.fhe_ntt_inverse(g.ctx, dev.data_ptr(), [i % level for i in range(limbs)], limbs)
    torch.cuda.synchronize()
    return dev.cpu().numpy().view(np.uint64)


def test_noalloc_matches_mod_switch_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_07308_gb300 import build

    build.build()
    from paper_2407_07308_gb300 import fhe
    from tests.gpu_setup import GpuSetup

    g = GpuSetup(seed=31, logN=14, p=131, L=10, K=3, **CHAIN50)
    try:
        N, L = g.N, g.L
        rnd = random.Random(5)
        # (count, npoly, level): two calls in a row, the scratch filled exactly
        # (32 two-poly ciphertexts at N = 2^14), and a three-poly tensor
        cases = [(3, 2, L), (5, 2, L - 3), (SCRATCH_WORDS // (2 * N), 2, L - 1), (4, 3, L - 2)]
        for call, (count, npoly, level) in enumerate(cases):
            rows = [[rnd.randrange(131) for _ in range(g.ns)] for _ in range(count)]
            ct = g.encrypt_slots(rows, seed=40 + call)
            if npoly == 3:
                ct = g.own(fhe.fhe_mul(g.ctx, ct, ct))
            if level < L:
                ct = g.own(fhe.fhe_mod_switch(g.ctx, ct, level))
            want = g.export(g.own(fhe.fhe_mod_switch(g.ctx, ct, level - 1)))
            dev_in = _to_device_ntt(fhe, g, g.export(ct), npoly, level)
            dev_out = torch.zeros((count, npoly, level - 1, N), dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            # no cached block left and the next allocation refused: a call that
            # allocated anything would fail
            fhe.fhe_ctx_sync(g.ctx)
            fhe.fhe_ctx_trim(g.ctx)
            fhe.fhe_ctx_memory_peak(g.ctx, reset=True)
            used = fhe.fhe_ctx_memory(g.ctx)[1]
            fhe.fhe_ctx_inject_alloc_failure(g.ctx, 0)
            try:
                fhe.fhe_mod_switch_noalloc(g.ctx, dev_in.data_ptr(), dev_out.data_ptr(), count, npoly, level)
                fhe.fhe_ctx_sync(g.ctx)
            finally:
                fhe.fhe_ctx_inject_alloc_failure(g.ctx, -1)
            assert fhe.fhe_ctx_memory(g.ctx)[1] == used
            assert fhe.fhe_ctx_memory_peak(g.ctx) == used
            got = _from_device_ntt(fhe, g, dev_out, npoly, level - 1)
            assert np.array_equal(got, want), f"call {call}"
            if npoly == 2:
                assert g.decrypt(ct).tolist() == rows
        # sizes beyond the fixed scratch are refused before any GPU work
        with pytest.raises(fhe.FheError) as ei:
            fhe.fhe_mod_switch_noalloc(g.ctx, dev_in.data_ptr(), dev_out.data_ptr(), SCRATCH_WORDS // N + 1, 2, L)
        assert ei.value.code == -1
    finally:
        g.close()
