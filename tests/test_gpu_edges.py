"""Edge cases on the GPU against the oracle: a single periodic element (every face its own
neighbour) in 2D and 3D, at N = 2, 3, 7; the free stream (a constant state, the method's
degenerate case) on the curved mesh, which every form must keep to rounding; zero steps."""
import numpy as np
import pytest

import cases
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg


def _single(dim, warp=0.0):
    def build(x):
        lo, hi = (-np.pi,) * dim, (np.pi,) * dim
        xyz, nbr, face = W.box_mesh((1,) * dim, x, lo, hi, periodic=True, warp=warp)
        if dim == 3:
            w = W.tgv_primitive(xyz, 1.4, 0.3)
        else:
            w = np.empty((1, 4, xyz.shape[2]))
            w[:, 0] = 1.0 + 0.2 * np.sin(xyz[:, 0])
            w[:, 1] = 0.3 * np.cos(xyz[:, 1])
            w[:, 2] = -0.2
            w[:, 3] = 1.0 + 0.1 * np.cos(xyz[:, 0] + xyz[:, 1])
        return xyz, nbr, face, w
    return build


def _rhs_pair(dg, pair, w_o, w_g):
    import torch
    u_o = pair.orc.prim_to_cons(w_o)
    r_o = pair.orc.rhs(u_o)
    pair.gpu.set_primitive(w_g)
    dt = torch.float32 if pair.gpu.precision == dg.DG_MIXED else torch.float64
    u_d = torch.empty(pair.gpu.shape, dtype=torch.float64, device="cuda")
    dg.dg_get_state(pair.gpu.ctx, u_d)
    u_d = u_d.to(dt)
    r_d = torch.empty_like(u_d)
    dg.dg_rhs(pair.gpu.ctx, u_d, r_d)
    dg.dg_sync(pair.gpu.ctx)
    return r_d.double().cpu().numpy(), r_o


SINGLE = [(3, 3, dict(equations=1, mu=0.02, Pr=0.72)), (3, 7, {}), (3, 2, dict(alpha_max=0.5)),
          (2, 3, dict(alpha_max=0.5)), (2, 7, {})]


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-4)])
@pytest.mark.parametrize("dim,N,kw", SINGLE)
def test_single_periodic_element(dg, precision, tol, dim, N, kw):
    p = cases.Pair(_single(dim), dim, N, precision=precision, **kw)
    try:
        w_o = cases.perturbed_state(p.mesh_o[3], 3, amp=0.05)
        w_g = cases.perturbed_state(p.mesh_g[3], 3, amp=0.05)
        r_g, r_o = _rhs_pair(dg, p, w_o, w_g)
        err = cases.field_errors(r_g, r_o, 1, dim)
        assert err.max() < tol, err
    finally:
        p.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", [{}, dict(equations=1, mu=0.02, Pr=0.72, alpha_max=0.5),
                                dict(volume_flux=5, surface_flux=3),
                                dict(equations=1, mu=0.02, Pr=0.72, sutherland_s=0.4042, sutherland_rt=0.7)])
def test_free_stream_on_the_curved_mesh(dg, precision, kw):
    """A constant state has zero right-hand side (the discrete metric identities): to FP64
    rounding in the FP64 form and to FP32 rounding in the mixed form, relative to the size
    of the flux differences it cancels."""
    import torch
    x, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face = W.box_mesh((3, 3, 3), x, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=0.15)
    s = dg.Solver(3, 3, xyz, nbr, face, precision=precision, **kw)
    try:
        w = np.broadcast_to(np.array([1.1, 0.3, -0.2, 0.5, 0.9])[None, :, None], (27, 5, 64)).copy()
        s.set_primitive(w)
        dt = torch.float32 if precision == 1 else torch.float64
        u = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(s.ctx, u)
        u = u.to(dt)
        r = torch.empty_like(u)
        dg.dg_rhs(s.ctx, u, r)
        dg.dg_sync(s.ctx)
        scale = float(u.abs().max()) * 10.0   # |f| times |Ja|/J ~ 1/h on this mesh
        eps = 1e-12 if precision == 0 else 2e-5
        assert float(r.abs().max()) < eps * scale
        if kw.get("alpha_max"):
            assert np.all(dg.dg_get_alpha(s.ctx, 27) == 0.0)
    finally:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_zero_steps_change_nothing(dg, precision):
    x, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face, w = cases.tgv(x, 2, warp=0.1)
    s = dg.Solver(3, 3, xyz, nbr, face, precision=precision)
    try:
        s.set_primitive(w)
        a, _ = s.get_state()
        assert s.step(0, cfl=0.5) == 0.0
        b, _ = s.get_state()
        assert np.array_equal(a, b)
    finally:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_unaligned_input_takes_the_per_thread_staging(dg, precision):
    """dg_rhs on a state that starts off a 16-byte boundary: the kernels check the address
    and stage with per-thread copies instead of bulk (TMA) copies; the result is the same
    bit for bit as from an aligned copy of the same state."""
    import torch
    x, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face, w = cases.tgv(x, 3, warp=0.1)
    s = dg.Solver(3, 3, xyz, nbr, face, precision=precision, equations=1, mu=0.02, Pr=0.72)
    try:
        s.set_primitive(cases.perturbed_state(w, 5))
        dt = torch.float32 if precision == 1 else torch.float64
        u64 = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(s.ctx, u64)
        u = u64.to(dt).contiguous()
        n = u.numel()
        buf = torch.empty(n + 1, dtype=dt, device="cuda")
        u_off = buf[1:].view(s.shape)          # 4 or 8 bytes past a 16-byte boundary
        u_off.copy_(u)
        assert u.data_ptr() % 16 == 0 and u_off.data_ptr() % 16 != 0
        r_a = torch.empty_like(u)
        r_b = torch.empty_like(u)
        dg.dg_rhs(s.ctx, u, r_a)
        dg.dg_rhs(s.ctx, u_off, r_b)
        dg.dg_sync(s.ctx)
        assert torch.equal(r_a, r_b)
    finally:
        s.close()


@pytest.mark.parametrize("where", ["pinned", "device"])
def test_state_conversion_odd_length_and_unaligned(dg, where):
    """The mixed form's state conversions (FP64 <-> FP32 pair) use 16-byte accesses for
    aligned buffers and the scalar path for the odd last value and for unaligned buffers:
    an odd-length state (3^3 elements at N = 2, 3645 values) gives the same bits through a
    16-byte aligned buffer and one 8 bytes off, and set / get returns the input to the
    pair's precision (|u - (hi + lo)| <= 2^-48 |u|)."""
    import torch
    p = cases.Pair(lambda x: cases.tgv(x, None, warp=0.1, shape=(3, 3, 3)), 3, 2,
                   precision=dg.DG_MIXED)
    try:
        u = p.orc.prim_to_cons(cases.perturbed_state(p.mesh_o[3], 5, amp=0.05))
        n = u.size
        assert n % 2 == 1
        dev = "cuda" if where == "device" else "cpu"

        def buf(off):
            b = torch.zeros(n + 2, dtype=torch.float64, device=dev)
            if where == "pinned":
                b = b.pin_memory()
            v = b[off:off + n].view(u.shape)
            assert v.data_ptr() % 16 == 8 * off
            return v

        outs = []
        for off in (0, 1):
            src = buf(off)
            src.copy_(torch.from_numpy(u))
            dg.dg_set_state(p.gpu.ctx, src)
            dst = buf(off)
            dg.dg_get_state(p.gpu.ctx, dst)
            torch.cuda.synchronize()
            outs.append(dst.cpu().numpy().copy())
        assert np.array_equal(outs[0], outs[1])
        assert np.abs(outs[0] - u).max() <= 2.0 ** -47 * np.abs(u).max()
    finally:
        p.close()
