"""mlmc_dk_run_level_static: the level batch for callers that cannot allocate
device memory when they run it (processes that serve all GPU memory from a
pool reserved at start-up, loops where cudaMalloc/cudaFree would synchronise
the device).  Its partial sums live in the library's statically allocated
device array instead of the context's scratch buffer.

Checked through the C-ABI against mlmc_dk_run_level_dev on the same inputs,
for several calls in a row: per-sample outputs identical, sums equal up to
FP64 summation order (the static array can hold fewer sample slots, which
changes only the order of the sums).  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2311_08872_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_08872_gb300 import build as libbuild
    libbuild.build()
    from paper_2311_08872_gb300 import mlmc_dk
    return mlmc_dk


def _run(ctx, dk, static, level, tag, first, count, seed):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    sums = torch.full((dk.sums_len(ctx.n_quant),), float("nan"), dtype=torch.float64, device="cuda")
    samp = torch.full((count, dk.sample_stride(ctx.n_obs)), float("nan"), dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    if static:
        ctx.run_level_static(level, tag, first, count, seed, sums.data_ptr(), samp.data_ptr(), err.data_ptr(), st)
    else:
        ctx.run_level_dev(level, tag, first, count, seed, sums.data_ptr(), samp.data_ptr(), st)
    torch.cuda.synchronize()
    return sums.cpu().numpy(), samp.cpu().numpy(), int(err.item())


@pytest.mark.parametrize("name,L_max,calls", [
    # two calls in a row on one context: a multi-warp coupled level, then a warp-resident level
    ("mlmc16_256", 2, [(2, 0, 10, 700, 5), (1, 0, 0, 5000, 6), (2, 1, 3, 300, 7)]),
    # 4^2 grids keep 32 samples per CTA: the static array limits the grid (fewer slots)
    ("paper_reg", 1, [(0, 0, 0, 300000, 8), (1, 0, 0, 50000, 9)]),
    # the same entry point on a theta-scheme context (Crank--Nicolson weights) ...
    ("theta16_64", 2, [(2, 0, 0, 600, 10), (1, 0, 4, 900, 11)]),
    # ... and on the Fourier coupling's ratio-3 hierarchy
    ("fourier6_54", 2, [(2, 0, 0, 400, 12), (1, 0, 2, 700, 13)]),
    # the cluster kernels: the 128^2 theta level (4-CTA clusters), the 162^2 Fourier level (6-CTA clusters)
    ("theta16_128", 3, [(3, 0, 0, 40, 14)]),
    ("fourier6_162", 3, [(3, 0, 5, 30, 15)]),
])
def test_static_scratch_matches_context_scratch(dk, name, L_max, calls):
    wl = W.get(name).with_(L_max=L_max)
    with dk.Context.from_workload(wl) as ctx:
        for level, tag, first, count, seed in calls:
            ref_sums, ref_samp, _ = _run(ctx, dk, False, level, tag, first, count, seed)
            got_sums, got_samp, err = _run(ctx, dk, True, level, tag, first, count, seed)
            assert err == 0
            assert np.array_equal(got_samp, ref_samp)
            assert got_sums[0] == ref_sums[0] == count
            assert got_sums[1] == ref_sums[1] == 0.0
            np.testing.assert_allclose(got_sums, ref_sums, rtol=1e-10, atol=1e-300)
