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
        for call, (count, level) in enumerate([(3, L), (5, L - 3)]):
            rows = [[rnd.randrange(131) for _ in range(g.ns)] for _ in range(count)]
            ct = g.encrypt_slots(rows, seed=40 + call)
            if level < L:
                ct = g.own(fhe.fhe_mod_switch(g.ctx, ct, level))
            want = g.export(g.own(fhe.fhe_mod_switch(g.ctx, ct, level - 1)))
            # the same ciphertext in caller-owned device memory, NTT domain
            coeff = g.export(ct)
            dev_in = torch.from_numpy(coeff.view(np.int64).copy()).cuda()
            limbs = count * 2 * level
            fhe.fhe_ntt_forward(g.ctx, dev_in.data_ptr(), [i % level for i in range(limbs)], limbs)
            dev_out = torch.zeros((count, 2, level - 1, N), dtype=torch.int64, device="cuda")
            torch.cuda.synchronize()
            fhe.fhe_mod_switch_noalloc(g.ctx, dev_in.data_ptr(), dev_out.data_ptr(), count, 2, level)
            fhe.fhe_ctx_sync(g.ctx)
            out_limbs = count * 2 * (level - 1)
            fhe.fhe_ntt_inverse(g.ctx, dev_out.data_ptr(), [i % (level - 1) for i in range(out_limbs)], out_limbs)
            torch.cuda.synchronize()
            got = dev_out.cpu().numpy().view(np.uint64)
            assert np.array_equal(got, want), f"call {call}"
            assert g.decrypt(ct).tolist() == rows
        # sizes beyond the fixed scratch are refused before any GPU work
        with pytest.raises(fhe.FheError) as ei:
            fhe.fhe_mod_switch_noalloc(g.ctx, dev_in.data_ptr(), dev_out.data_ptr(), 64, 2, L)
        assert ei.value.code == -1
    finally:
        g.close()
