"""ssh_hash_device_noalloc: the hashing entry point for callers that cannot call
cudaMalloc (its working buffers live in a fixed device array of the library).
Its outputs must equal those of the allocating entry point ssh_hash_device --
sketch bits, shingle sets, minhashes and bucket keys are integers, so equal
means bit for bit -- on consecutive calls, since every call reuses the same
array and starts from whatever the previous call left there.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import re

import numpy as np
import pytest

from paper_1610_07328_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CFG_SCALE = dict(W=80, delta=3, n=15, K=4, L=25, band=0.05, seed=0)   # m = 512
CFG_TINY = dict(W=32, delta=3, n=8, K=4, L=16, band=0.05, seed=0)     # m = 128


def _outputs(binding, idx, d_x, m, noalloc):
    N = d_x.shape[0]
    nb = (m - idx.W) // idx.delta + 1
    S = nb - idx.n + 1
    KL = idx.K * idx.L
    out = dict(bits=torch.full((N, (nb + 31) // 32), -1, dtype=torch.int32, device="cuda"),
               ids=torch.full((N, S), -1, dtype=torch.int32, device="cuda"),
               cnt=torch.full((N, S), -1, dtype=torch.int32, device="cuda"),
               nnz=torch.full((N,), -1, dtype=torch.int32, device="cuda"),
               ks=torch.full((N, KL), -1, dtype=torch.int32, device="cuda"),
               ts=torch.full((N, KL), -1, dtype=torch.int32, device="cuda"),
               keys=torch.zeros((idx.L, N), dtype=torch.int64, device="cuda"))
    fn = binding.ssh_hash_device_noalloc if noalloc else binding.ssh_hash_device
    fn(idx.handle, d_x, m, N, out["bits"], out["ids"], out["cnt"], out["nnz"], out["ks"], out["ts"], out["keys"])
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    # shingle slots past each series' nnz are left untouched by both entry points
    for i, k in enumerate(res["nnz"]):
        res["ids"][i, k:] = -1
        res["cnt"][i, k:] = -1
    return res


@pytest.mark.parametrize("cfg,m,N,seed", [(CFG_SCALE, 512, 4000, 1), (CFG_TINY, 128, 3000, 2)])
def test_noalloc_hash_equals_allocating_hash_twice(cfg, m, N, seed):
    from paper_1610_07328_gb300 import binding
    with binding.SSHIndex(**cfg) as idx:
        x = synth.random_walk(N, m, seed=seed)
        d_x = torch.from_numpy(x).cuda()
        want = _outputs(binding, idx, d_x, m, noalloc=False)
        for call in range(2):  # the second call starts from the first call's leftovers
            got = _outputs(binding, idx, d_x, m, noalloc=True)
            for name in want:
                assert np.array_equal(got[name], want[name]), f"{name} differs on call {call}"
        # a different batch through the same scratch right after
        y = synth.ecg_like(1500, m, seed=seed + 10)
        d_y = torch.from_numpy(y).cuda()
        want_y = _outputs(binding, idx, d_y, m, noalloc=False)
        got_y = _outputs(binding, idx, d_y, m, noalloc=True)
        for name in want_y:
            assert np.array_equal(got_y[name], want_y[name]), f"{name} differs on the second batch"


def test_noalloc_rejects_counts_beyond_the_fixed_scratch():
    from paper_1610_07328_gb300 import binding
    with binding.SSHIndex(**CFG_SCALE) as idx:
        m, N = 512, 40_000  # more than the 16 MiB scratch holds at this shape
        d_x = torch.zeros((N, m), dtype=torch.float32, device="cuda")
        keys = torch.zeros((idx.L, N), dtype=torch.int64, device="cuda")
        with pytest.raises(binding.SSHError) as e:
            binding.ssh_hash_device_noalloc(idx.handle, d_x, m, N, d_keys=keys)
        assert e.value.status == binding.SSH_EINVAL
        assert "scratch" in str(e.value) and "at most" in str(e.value)
        assert (keys.cpu().numpy() == 0).all()  # nothing ran
        # the limit the message reports is exact: that many series fit, one more does not
        fit = int(re.search(r"at most (\d+) series", str(e.value)).group(1))
        assert 0 < fit < N
        binding.ssh_hash_device_noalloc(idx.handle, d_x[:fit], m, fit, d_keys=keys[:, :fit].contiguous())
        torch.cuda.synchronize()
        with pytest.raises(binding.SSHError) as e2:
            binding.ssh_hash_device_noalloc(idx.handle, d_x[:fit + 1], m, fit + 1,
                                            d_keys=keys[:, :fit + 1].contiguous())
        assert e2.value.status == binding.SSH_EINVAL
