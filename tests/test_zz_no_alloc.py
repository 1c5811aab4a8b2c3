"""er_solve_noalloc through the C ABI: the FP64 solve whose workspace is a fixed static
device array, for callers that cannot allocate device memory at solve time.  Two calls
in a row must match er_solve (same kernels and tiling, so the same iterates), neither may
change the device's free memory (the array is committed when the grid is created), and an
oversized request must be rejected.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def er():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_05818_gb300 import er as mod
    return mod


def test_noalloc_solve_matches_er_solve_twice(er):
    from paper_2607_05818_gb300 import instances as I
    inst = I.tiny_plain()
    k, seed = 128, 20260701
    g = er.grid_create(inst)
    Yt = torch.empty((inst.n, k), dtype=torch.float64, device="cuda")
    Z_ref = torch.empty_like(Yt)
    er.sketch(g, k, seed, "fp64", Yt)
    _, st_ref = er.solve(g, Yt, Z_ref, k, "fp64")
    torch.cuda.synchronize()
    ref = Z_ref.cpu().numpy()
    scale = np.maximum(np.abs(ref).max(axis=0), 1e-300)
    stream = torch.cuda.current_stream().cuda_stream
    Zs = [torch.full_like(Yt, float("nan")) for _ in range(2)]   # outputs allocated up front
    torch.cuda.synchronize()
    for call in range(2):
        Z = Zs[call]
        stats = er.er_solve_stats()
        free_before = torch.cuda.mem_get_info()[0]
        status = er._lib.er_solve_noalloc(g.handle, Yt.data_ptr(), Z.data_ptr(), k, None, ctypes.byref(stats),
                                          stream)
        assert status == er.ER_OK, (call, er.status_str(status), er._lib.er_last_error())
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        # no device allocation: any cudaMalloc moves the free figure by at least a 2 MiB page
        assert free_before - free_after < (1 << 20), (call, free_before, free_after)
        got = Z.cpu().numpy()
        assert np.max(np.abs(got - ref) / scale) <= 1e-9, call
        assert stats.iterations == st_ref["iterations"] and stats.converged_cols == k
    # beyond the static workspace: rejected before any launch
    Ybig = torch.zeros((inst.n, 132), dtype=torch.float64, device="cuda")
    Zbig = torch.zeros_like(Ybig)
    status = er._lib.er_solve_noalloc(g.handle, Ybig.data_ptr(), Zbig.data_ptr(), 132, None, None, stream)
    assert status == er.ER_ERR_INVALID_ARG
    assert b"262144" in er._lib.er_last_error()
    g.destroy()
