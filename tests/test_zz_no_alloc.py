"""The entry point that allocates nothing (mstopo_apply_K_f32_noalloc).

Some callers cannot call cudaMalloc: their device memory belongs to another allocator or a
fixed arena, or they may not trigger the device-wide synchronisation an allocation can
cause.  This entry point gives them the FP32 matrix-free matvec without a handle, using a
fixed static device array as work space.  It must agree with the handle-based entry point
mstopo_apply_K(..., MSTOPO_MIXED, ...) on the same inputs, on consecutive calls (the work
space is shared between calls).  Collected last so that a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matvec_matches_handle_matvec_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_3923_gb300 as m
    import workloads

    lib = m.load()
    wl = workloads.small(96, 40, seed=21, kind="voids", H=8, n_eig=4)
    prob = m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                     penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision="mixed")
    prob.set_design(torch.from_numpy(wl.rho).cuda(), wl.rmin, wl.beta, wl.etas, wl.cell)
    E32 = prob.get_field(m.FIELD_YOUNG, 0).float().contiguous()
    fixed = torch.from_numpy(np.ascontiguousarray(wl.fixed, dtype=np.uint8)).cuda()
    for call in range(2):
        u = torch.randn((wl.nely + 1, wl.nelx + 1, 2), dtype=torch.float64, device="cuda",
                        generator=torch.Generator(device="cuda").manual_seed(100 + call))
        y_ref = prob.apply_K(u, 0, m.MIXED)
        y = torch.full_like(u, float("nan"))
        st = lib.mstopo_apply_K_f32_noalloc(u.data_ptr(), y.data_ptr(), E32.data_ptr(),
                                            fixed.data_ptr(), wl.nelx, wl.nely, wl.nu, None)
        assert st == 0
        # same kernels on the same FP32 inputs: identical up to FP32 rounding (here exact)
        scale = float(y_ref.abs().max())
        assert float((y - y_ref).abs().max()) <= 2e-6 * scale


def test_noalloc_rejects_meshes_above_its_fixed_capacity():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_3923_gb300 as m
    lib = m.load()
    dummy = ctypes.c_void_p(1)   # never dereferenced: the size check comes first
    st = lib.mstopo_apply_K_f32_noalloc(dummy, dummy, dummy, dummy, 2048, 1024, 0.3, None)
    assert st == 1   # MSTOPO_INVALID_ARG: 2*2049*1025 DOFs > 2^22
    # the largest int32 sizes: the DOF count is formed in 64 bits and rejected, not wrapped
    st = lib.mstopo_apply_K_f32_noalloc(dummy, dummy, dummy, dummy, 2**31 - 1, 2**31 - 1, 0.3, None)
    assert st == 1
