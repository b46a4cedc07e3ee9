"""What the trained networks gain over the method without them, on the same GB300 and the
same state: the learned chemistry source against the plain FP64 source (device time per
evaluation, and the learned values' error against the plain ones), the corrected learned
source over a run (time per step, and the end state's error against the FP64 form), and the learned
temperature solve against the plain Newton iteration (device time per launch, and T
against the oracle's Newton solve).  Both networks are trained here by libdg's kernels
on states of the plain solver's own run (a 24 x 24 x 8 O-grid, N = 4: 576,000 nodes)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# stated accuracy of the learned source at the evaluation timed here: relative L2 over the
# nodes of S_learned - S_plain per species, over the norm of S_plain
SOURCE_L2_BAR = 0.1
# the temperature target of the learned form: max relative error against Newton
T_REL_BAR = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_17551_gb300 as dg
    dg.lib()
    return dg, torch


def _mesh(dg, react, precision=None):
    import workloads as W
    N = 4
    xi, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face = W.ogrid_mesh(xi, 24, 24, 8)
    vel = (2400.0 if react else 2000.0, 0.0, 0.0)
    hot = (1.2, 3000.0) if react else None
    w0 = W.mixture_primitive(xyz, rho=0.1, vel=vel, T=300.0, seed=7, cylinder=0.5, hot=hot)
    fs = W.mixture_primitive(xyz[:1], rho=0.1, vel=vel, T=300.0, seed=7)[0, :, 0]
    s = dg.Solver(3, N, xyz, nbr, face, n_species=5, species=W.species_table(),
                  volume_flux=dg.DG_VF_DUCROS, surface_flux=dg.DG_SF_LLF, bc_kind=[1, 2, 3],
                  bc_prim=np.stack([fs] * 3), alpha_max=0.5,
                  precision=dg.DG_MIXED if precision is None else precision,
                  reactions=W.reaction_table() if react else None)
    s.set_primitive(w0)
    return s, w0, xyz, nbr, face


def _record(name, d):
    out = os.environ.get("DG_GAIN_LOG")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps({name: d}) + "\n")


def test_learned_source_gain(env):
    dg, torch = env
    from paper_2511_17551_gb300 import surrogate as S
    s, w0, *_ = _mesh(dg, True)
    try:
        X, Y = S.collect_source(s.ctx, 200_000, 8, 1, cfl=0.05)
        params, stats, hist = S.train_source(X, Y, epochs=20, batch=4096, lr=2e-3)
        s.set_primitive(w0)
        u = torch.empty(s.shape, dtype=torch.float64, device="cuda")
        dg.dg_get_state(s.ctx, u)
        u32 = u.float()
        r = torch.empty_like(u32)

        def timed(n=5):
            dg.dg_rhs(s.ctx, u32, r)  # warm
            dg.dg_sync(s.ctx)
            dg.dg_profile(s.ctx, 1)
            dg.dg_profile_read(s.ctx)
            for _ in range(n):
                dg.dg_rhs(s.ctx, u32, r)
            p = dg.dg_profile_read(s.ctx)
            dg.dg_profile(s.ctx, 0)
            src, _, _ = dg.dg_get_source(s.ctx, s.shape)
            return p["chem"][0] / p["chem"][1], src

        plain_ms, S_plain = timed()
        dg.dg_set_surrogate(s.ctx, params, stats, which=dg.DG_SURROGATE_SOURCE)
        dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        learned_ms, S_l = timed()
        acc, fb = dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        num = np.linalg.norm((S_l - S_plain).transpose(1, 0, 2).reshape(5, -1), axis=1)
        den = np.linalg.norm(S_plain.transpose(1, 0, 2).reshape(5, -1), axis=1)
        l2 = num / den
        rec = {"plain_ms": plain_ms, "learned_ms": learned_ms, "gain": plain_ms / learned_ms,
               "accepted_fraction": acc / max(1, acc + fb), "l2_per_species_vs_plain": l2.tolist()}
        print("learned source:", rec)
        _record("source", rec)
        assert learned_ms < plain_ms, rec
        assert l2.max() < SOURCE_L2_BAR, rec
    finally:
        s.close()


# the corrected learned source over a run: per-field relative L2 of the end state against
# the FP64 form's plain run (the stated bar of the mixed form with learned parts)
RUN_STEPS = 50
RUN_L2_BAR = 1e-5


def _l2(a, ref):
    mom = np.linalg.norm(ref[:, 5:8])
    return np.array([np.linalg.norm(a[:, v] - ref[:, v]) / (mom if 5 <= v < 8 else np.linalg.norm(ref[:, v]))
                     for v in range(a.shape[1])])


def test_corrected_source_run_gain(env):
    """RUN_STEPS CK45 steps of the reacting O-grid (CFL 0.05): the mixed form with the plain
    source against the mixed form with the corrected learned source (tolerance 0.002, a
    refresh every step), both against the FP64 form's plain run.  The corrected run is
    faster than the plain mixed run and within RUN_L2_BAR on every conserved field."""
    dg, torch = env
    import time
    from paper_2511_17551_gb300 import surrogate as S
    s64, w0, *_ = _mesh(dg, True, dg.DG_FP64)
    try:
        s64.step(RUN_STEPS, 0.05)
        u64, _ = s64.get_state()
    finally:
        s64.close()
    s, w0, *_ = _mesh(dg, True)
    try:
        def run():
            s.set_primitive(w0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(RUN_STEPS, 0.05)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) * 1e3 / RUN_STEPS, s.get_state()[0]
        run()  # warm
        plain_ms, u_plain = run()
        s.set_primitive(w0)
        X, Y = S.collect_source(s.ctx, 500_000, 8, max(1, RUN_STEPS // 8), cfl=0.05)
        params, stats, hist = S.train_source(X, Y, epochs=60, batch=4096, lr=3e-3, lr_final=1e-4)
        st = stats.copy()
        st[50] = st[51] = 0.002
        dg.dg_set_surrogate(s.ctx, params, st, which=dg.DG_SURROGATE_SOURCE)
        dg.dg_set_source_refresh(s.ctx, 1)
        dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        corr_ms, u_c = run()
        acc, fb = dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        rec = {"steps": RUN_STEPS, "plain_mixed_ms_per_step": plain_ms, "corrected_ms_per_step": corr_ms,
               "gain": plain_ms / corr_ms, "accepted_fraction": acc / max(1, acc + fb),
               "l2_plain_mixed_vs_fp64": _l2(u_plain, u64).tolist(),
               "l2_corrected_vs_fp64": _l2(u_c, u64).tolist()}
        print("corrected source run:", rec)
        _record("corrected_run", rec)
        assert corr_ms < plain_ms, rec
        assert _l2(u_c, u64).max() < RUN_L2_BAR, rec
    finally:
        s.close()


def test_learned_temperature_gain(env):
    dg, torch = env
    import oracle
    import workloads as W
    from paper_2511_17551_gb300 import surrogate as S
    s, w0, xyz, nbr, face = _mesh(dg, False)
    try:
        X, T = S.collect(s.ctx, 200_000, 10, 2, cfl=0.3)
        params, stats, hist = S.train(X, T, epochs=20, batch=4096, lr=2e-3)
        shape = (s.K, s.np)
        s.set_primitive(w0)
        dg.dg_profile(s.ctx, 1)
        dg.dg_profile_read(s.ctx)
        s.set_primitive(w0)  # resets the temperature cache: the next solve starts cold
        T_cold = dg.dg_get_temperature(s.ctx, shape)
        cold = dg.dg_profile_read(s.ctx)["thermo"][0]
        dg.dg_get_temperature(s.ctx, shape)
        warm = dg.dg_profile_read(s.ctx)["thermo"][0]
        dg.dg_set_surrogate(s.ctx, params, stats)
        dg.dg_surrogate_stats(s.ctx)
        s.set_primitive(w0)
        dg.dg_profile_read(s.ctx)
        T_mlp = dg.dg_get_temperature(s.ctx, shape)
        mlp = dg.dg_profile_read(s.ctx)["thermo"][0]
        acc, fb = dg.dg_surrogate_stats(s.ctx)
        dg.dg_profile(s.ctx, 0)
        # the oracle's Newton temperature of the same primitive state
        N = 4
        xo, _ = oracle.lgl(N)
        xyz_o, nbr_o, face_o = W.ogrid_mesh(xo, 24, 24, 8)
        w_o = W.mixture_primitive(xyz_o, rho=0.1, vel=(2000.0, 0.0, 0.0), T=300.0, seed=7, cylinder=0.5)
        o = oracle.Oracle(3, N, xyz_o, nbr_o, face_o, n_species=5, species=W.species_table(), volume_flux=1)
        T_o = o.temperature(o.prim_to_cons(w_o))
        rel = float(np.abs(T_mlp / T_o - 1).max())
        rec = {"cold_newton_ms": cold, "converged_cache_newton_ms": warm, "surrogate_ms": mlp,
               "gain_vs_cold": cold / mlp, "gain_vs_converged_cache": warm / mlp,
               "accepted_fraction": acc / max(1, acc + fb), "max_rel_T_vs_oracle_newton": rel,
               "max_rel_T_plain_vs_oracle_newton": float(np.abs(T_cold / T_o - 1).max())}
        print("learned temperature:", rec)
        _record("temperature", rec)
        assert rel < T_REL_BAR, rec
    finally:
        s.close()
