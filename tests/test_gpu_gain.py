"""What the trained networks gain over the method without them, on the same GB300 and the
same state: the learned chemistry source against the plain FP64 source (device time per
evaluation, and the learned values' error against the plain ones), and the learned
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


def _mesh(dg, react):
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
                  bc_prim=np.stack([fs] * 3), alpha_max=0.5, precision=dg.DG_MIXED,
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
