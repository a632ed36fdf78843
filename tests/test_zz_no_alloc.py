"""The projection entry point that allocates nothing.

Callers that may not allocate device memory while they run (a real-time
pipeline that reserved all device memory at start-up, a plugin whose host
application's pool owns the device) use smre_dykstra_project_static, which
keeps every intermediate buffer in the library's static 16 MiB device array.
It must give the same image as the handle-based smre_dykstra_project, on
repeated calls too (the array keeps the previous call's contents), and must
turn away sizes that do not fit.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _err(a, ref):
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.abs(a - ref).max() / np.abs(ref).max())


def test_static_entry_point_matches_allocating_path_twice(torch_cuda):
    import paper_1503_03492_gb300 as smre
    from synthetic import emitter_residual

    H, W, sides = 96, 80, [1, 2, 3, 4]
    cS = smre.smre_bounds(smre.make_params(H, W, sides, alpha=0.9))
    kw = dict(cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS, max_cycles=25, tol=-1.0)
    stream = torch_cuda.cuda.current_stream()
    for call, seed in enumerate((11, 12)):
        x0 = np.ascontiguousarray(emitter_residual(H, W, n_emitters=12, seed=seed), np.float32)
        xd = torch_cuda.from_numpy(x0).cuda()
        ref = torch_cuda.empty_like(xd)
        with smre.Projector(H, W, sides, stream=stream, **kw) as P:
            r_ref = P.project(xd, ref)
        out = torch_cuda.full_like(xd, float("nan"))
        p = smre.make_params(H, W, sides, **kw)
        r = smre.smre_dykstra_project_static(p, xd, out, stream=stream)
        assert r.cycles == r_ref.cycles == 25, (call, r.cycles, r_ref.cycles)
        e = _err(out.cpu().numpy(), ref.cpu().numpy())
        assert e <= TOL, (call, e)
        # and against the FP64 oracle directly, at the same bar
        import oracle
        o = oracle.dykstra(x0.astype(np.float64), sides, list(cS), max_cycles=25, tol=-1).x
        e64 = _err(out.cpu().numpy(), o)
        assert e64 <= TOL, (call, e64)


def test_static_entry_point_allocates_nothing_after_warm_up(torch_cuda):
    """After one warm-up call (which makes the runtime load the library's
    device code, the static array with it), further calls leave the device's
    free memory unchanged; host images work too."""
    import paper_1503_03492_gb300 as smre
    from synthetic import emitter_residual

    H, W, sides = 64, 72, [1, 2, 4]
    cS = smre.smre_bounds(smre.make_params(H, W, sides, alpha=0.9))
    kw = dict(cmode=smre.SMRE_C_EXPLICIT, c_explicit=cS, max_cycles=10, tol=-1.0)
    p = smre.make_params(H, W, sides, **kw)
    x0 = np.ascontiguousarray(emitter_residual(H, W, n_emitters=8, seed=21), np.float32)
    out = np.empty_like(x0)
    smre.smre_dykstra_project_static(p, x0, out)          # warm-up (host images)
    torch_cuda.cuda.synchronize()
    free0 = torch_cuda.cuda.mem_get_info()[0]
    out2 = np.full_like(x0, np.nan)
    r = smre.smre_dykstra_project_static(p, x0, out2)
    torch_cuda.cuda.synchronize()
    assert torch_cuda.cuda.mem_get_info()[0] == free0
    assert r.cycles == 10
    with smre.Projector(H, W, sides, **kw) as P:
        ref = np.empty_like(x0)
        P.project(x0, ref)
    assert _err(out2, ref) <= TOL
    assert np.array_equal(out, out2)


def test_static_entry_point_rejects_sizes_beyond_its_buffer(torch_cuda):
    import paper_1503_03492_gb300 as smre

    H = W = 1024
    x = torch_cuda.zeros(H, W, device="cuda")
    p = smre.make_params(H, W, list(range(1, 9)), max_cycles=2)
    with pytest.raises(smre.SmreError) as ei:
        smre.smre_dykstra_project_static(p, x, x)
    assert ei.value.status == smre.SMRE_EINVAL
    assert "static buffer" in str(ei.value)
