"""Benchmark: DOF x RHS-evaluations per second of the entropy-stable DGSEM on GB300.

Workload (default): Navier-Stokes Taylor-Green vortex, Re = 1600, Pr = 0.72, Ma = 0.1,
32^3 curved hexahedra (x_i += 0.1 sin x sin y sin z), degree N = 3, seeded synthetic
initial state.  One step = one Carpenter-Kennedy RK45 step (5 right-hand sides) at
CFL 0.5 with the time step reduced on the device.  ``value`` is the mixed form
(FP32 fluxes / sums, FP64 reductions); the FP64 form is timed beside it.

Arms: ``--impl ours`` (default) runs libdg; ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
Multi-GPU: N > 1 runs independent replicas of the workload, one per rank (weak scaling,
no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

CONFIGS = {
    "tgv_ns_32^3_N3": dict(n_el=32, N=3, warp=0.1, mu=1.0 / 1600.0),
    "tgv_ns_16^3_N7": dict(n_el=16, N=7, warp=0.1, mu=1.0 / 1600.0),
    "tgv_euler_4^3_N3": dict(n_el=4, N=3, warp=0.0, mu=0.0),
    # profiling case for ncu section captures: same kernels, 245 MB working set (> L2)
    "tgv_ns_24^3_N3": dict(n_el=24, N=3, warp=0.1, mu=1.0 / 1600.0),
}
# algorithmic HBM words per node of one RK-stage launch of the method (unique bytes,
# neighbour traces excluded): the main kernel reads u, du, the metric terms Ja and 1/J
# and the 12 viscous words, and writes du and the new u (5 + 5 + 9 + 1 + 12 + 5 + 5 = 42
# words = 168 B in FP32 with NS; 30 words = 120 B for Euler).  The compensated FP32 state
# adds its low part u_lo, read and written (10 words = 40 B): an implementation choice of
# the mixed form, reported beside the method's bytes, not in them.  The gradient kernel
# reads u, Ja, 1/J and writes the viscous fluxes.
WORDS_MAIN_NS = 5 + 5 + 9 + 1 + 12 + 5 + 5
WORDS_MAIN_EULER = 5 + 5 + 9 + 1 + 5 + 5
WORDS_COMPENSATION = 10
WORDS_GRAD = 5 + 9 + 1 + 12
# dram__bytes_read.sum + dram__bytes_write.sum per node of one launch of the current
# mixed-form NS N=3 rhs_kernel on the full 32^3 workload (one ncu capture, one pass:
# 271,931,392 B read + 95,960,832 B written over 2,097,152 nodes)
RHS_DRAM_B_PER_NODE = 176.64
# FP64 flops per node of the FP64-form NS N=3 rhs_kernel (2 DFMA + DMUL + DADD thread
# instructions, one ncu capture of the 16^3 case): its roofline is the FP64 pipe
RHS_FP64_FLOPS_PER_NODE = 1005.3


def job_rate(ms_local, units_local, world, device="cpu"):
    """Whole-job throughput of N replicas: the units all ranks processed over the slowest
    rank's time (max over ranks of the timed region).  Returns (units/s, max ms)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return world * units_local / (ms * 1e-3), ms


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler during the timed region (200 ms)."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nme, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(nme)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def build_workload(cfg, xi):
    xyz, nbr, face = W.box_mesh((cfg["n_el"],) * 3, xi, (-np.pi,) * 3, (np.pi,) * 3,
                                periodic=True, warp=cfg["warp"])
    return xyz, nbr, face, W.tgv_primitive(xyz)


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import paper_2511_17551_gb300 as dg

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    cfg = CONFIGS[args.config]
    N = cfg["N"]
    xi, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face, w0 = build_workload(cfg, xi)
    K, npn = xyz.shape[0], (N + 1) ** 3
    dof = K * npn * 5
    eq = dg.DG_NAVIER_STOKES if cfg["mu"] > 0 else dg.DG_EULER
    stream = torch.cuda.current_stream()

    def make(precision):
        # p_ref = the mean pressure p0 = 1/(gamma Ma^2) of the Mach-0.1 state
        s = dg.Solver(3, N, xyz, nbr, face, equations=eq, mu=cfg["mu"], Pr=0.72,
                      precision=precision, stream=stream.cuda_stream, p_ref=1.0 / (1.4 * 0.01))
        s.set_primitive(w0)
        return s

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(s, steps, profile=False):
        s.step(args.warmup, cfg_cfl)
        if profile:
            dg.dg_profile(s.ctx, 1)
            dg.dg_profile_read(s.ctx)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        s.step(steps, cfg_cfl)
        t1.record(stream)
        barrier()
        ms = t0.elapsed_time(t1)
        prof = dg.dg_profile_read(s.ctx) if profile else None
        if profile:
            dg.dg_profile(s.ctx, 0)
        return ms, prof

    cfg_cfl = 0.5
    # --- mixed form: the headline
    s = make(dg.DG_MIXED)
    clocks = Clocks(local_rank)
    ms, prof = timed_steps(s, args.steps, profile=True)
    clk = clocks.stop()
    value, ms = job_rate(ms, dof * 5 * args.steps, world, device="cuda")
    # --- end to end through the C ABI with host buffers (pinned), copies inside the region
    u_host = torch.empty((K, 5, npn), dtype=torch.float64).pin_memory()
    dg.dg_get_state(s.ctx, u_host)
    e2e_steps = max(1, min(args.steps, 10))
    barrier()
    t_start = time.perf_counter()
    for _ in range(e2e_steps):
        dg.dg_set_state(s.ctx, u_host)
        dg.dg_step_rk(s.ctx, 1, cfg_cfl)
        dg.dg_get_state(s.ctx, u_host)
    barrier()
    e2e_s = time.perf_counter() - t_start
    e2e_value = world * dof * 5 * e2e_steps / e2e_s
    # where the end-to-end time goes (each call synchronises): host wall ms per call
    parts = {"set_state": 0.0, "step": 0.0, "get_state": 0.0}
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        dg.dg_set_state(s.ctx, u_host)
        t1 = time.perf_counter()
        dg.dg_step_rk(s.ctx, 1, cfg_cfl)
        t2 = time.perf_counter()
        dg.dg_get_state(s.ctx, u_host)
        t3 = time.perf_counter()
        parts["set_state"] += (t1 - t0) * 1e3 / e2e_steps
        parts["step"] += (t2 - t1) * 1e3 / e2e_steps
        parts["get_state"] += (t3 - t2) * 1e3 / e2e_steps
    s.close()
    # --- FP64 form on the same GPU
    s64 = make(dg.DG_FP64)
    k64 = max(1, min(args.steps, 5))
    ms64, prof64 = timed_steps(s64, k64, profile=True)
    s64.close()
    value64 = world * dof * 5 * k64 / (ms64 * 1e-3)

    # roofline of the dominant kernel (main RHS / RK-stage kernel of the mixed form)
    peak, peak_kind = _peaks()
    fp64_peak = dg.dg_peak_flops(dg.DG_FP64, 4000)
    fp32_peak = dg.dg_peak_flops(dg.DG_MIXED, 20000)
    rhs64_ms = prof64["rhs"][0] / max(1, prof64["rhs"][1])
    fp64_achieved = RHS_FP64_FLOPS_PER_NODE * K * npn / (rhs64_ms * 1e-3) / 1e12
    rhs_ms, rhs_n = prof["rhs"]
    words = WORDS_MAIN_NS if eq == dg.DG_NAVIER_STOKES else WORDS_MAIN_EULER
    bytes_launch = words * 4 * K * npn
    achieved = bytes_launch / (rhs_ms / rhs_n * 1e-3) / 1e9
    moved = (words + WORDS_COMPENSATION) * 4 * K * npn / (rhs_ms / rhs_n * 1e-3) / 1e9
    launches = sum(n for _, n in prof.values())
    out = {
        "metric": "DOF*RHS-evals/s (FP32+FP64-reductions form; FP64 form beside it)",
        "value": value, "unit": "DOF*RHS/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.config, "elements": K, "N": N, "dof": dof,
                   "rk": "CK45 5-stage, CFL 0.5, device dt", "parallelism": "replicas",
                   "l2_flush": "working set %.0f MB > L2 (129 MB)" % (
                       (words + WORDS_COMPENSATION + WORDS_GRAD) * 4 * K * npn / 1e6)},
        "fp64_form": {"value": value64, "ms_per_step": ms64 / k64, "steps": k64,
                      "rhs_kernel_ms": rhs64_ms,
                      "roofline": None if not (eq == dg.DG_NAVIER_STOKES and N == 3) else
                                  {"bound": "alu", "achieved": fp64_achieved, "peak": fp64_peak,
                                   "unit": "TFLOP/s", "frac": fp64_achieved / fp64_peak,
                                   "flops_per_node": RHS_FP64_FLOPS_PER_NODE,
                                   "peak_source": "FP64 FMA chains measured here (dg_peak_flops)"}},
        "e2e": {"value": e2e_value, "unit": "DOF*RHS/s", "h2d_bytes_per_step": dof * 8,
                "d2h_bytes_per_step": dof * 8,
                "host_ms_per_call": {k: round(v, 4) for k, v in parts.items()}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (RHS_DRAM_B_PER_NODE * K * npn
                                 if RHS_DRAM_B_PER_NODE and eq == dg.DG_NAVIER_STOKES and N == 3
                                 else None),
                     "kernel": "rhs_kernel<3,%d,1,NS> f32" % N,
                     "algorithmic_bytes_per_node": words * 4,
                     "ms_per_launch": rhs_ms / rhs_n,
                     "with_compensation": {"bytes_per_node": (words + WORDS_COMPENSATION) * 4,
                                           "achieved": moved, "frac": moved / peak},
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, burst copy)"},
        "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]}
                    for k, v in prof.items() if v[1]},
        "gpu_launches": launches,
        "clocks": clk,
    }
    out["arith_peaks_tflops"] = {"fp64_fma": fp64_peak, "fp32_fma": fp32_peak,
                                 "source": "measured here, FMA chains, 152x8 CTAs"}
    out["mlp_forward"] = run_mlp_forward()
    surrogate_T = None
    if not args.no_mixture:
        out["mixture"] = run_mixture(args, stream.cuda_stream, world, fp64_peak)
        surrogate_T = out["mixture"].pop("_surrogate")
    if not args.no_reacting:
        out["reacting"] = run_reacting(args, stream.cuda_stream, world, fp64_peak)
    if not args.no_other_shapes:
        out.update(run_other_shapes(args, stream.cuda_stream, world))
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"], r_oracle, u_oracle, n_or, dt_or, floors = cpu_baseline(cfg, args.cpu_seconds)
            floor, floor32, u_init_or = floors
            # both GPU forms against what the baseline leg computed: the state after the
            # same CK45 steps, and the right-hand side of the initial state
            par = {"norm": "relative L2 per conserved field (rho, rho v x3, rho E); momentum "
                           "over the momentum-block norm",
                   "steps": n_or, "dt": dt_or,
                   "note": "d(rho)/dt of the initial Taylor-Green state vanishes analytically "
                           "(uniform rho, solenoidal v): its relative RHS error divides by a "
                           "discretisation-error-sized norm; at Mach 0.1 the pressure p0 = 71 "
                           "cancels to gradients of order 0.1, so every right-hand-side "
                           "comparison sits on the rounding floor in rhs_oracle_ulp_floor",
                   "rhs_oracle_ulp_floor": floor, "rhs_oracle_fp32_ulp_floor": floor32,
                   "increment_note": "relative L2 per field of the increment u_n - u_0 over the steps "
                                     "against the oracle's increment (the state error divides by the "
                                     "state's norm, the increment error by the change's)"}
            for name, prec in (("fp64", dg.DG_FP64), ("mixed", dg.DG_MIXED)):
                sp = make(prec)
                ud = torch.empty(sp.shape, dtype=torch.float64, device="cuda")
                dg.dg_get_state(sp.ctx, ud)
                ud = ud.to(torch.float32 if prec == dg.DG_MIXED else torch.float64)
                rd = torch.empty_like(ud)
                dg.dg_rhs(sp.ctx, ud, rd)
                dg.dg_sync(sp.ctx)
                par["rhs_" + name] = field_errors(rd.double().cpu().numpy(), r_oracle)
                u0_g = sp.get_state()[0]
                sp.step(n_or, dt_fixed=dt_or)
                un_g = sp.get_state()[0]
                par["state_after_steps_" + name] = field_errors(un_g, u_oracle)
                par["increment_after_steps_" + name] = field_errors(un_g - u0_g, u_oracle - u_init_or)
                sp.close()
            out["parity_vs_oracle"] = par
            if not args.no_mixture:
                out["mixture"]["T_max_rel_vs_oracle_newton_initial_state"] = mixture_T_vs_oracle(args, surrogate_T)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_mlp_forward(n=4_608_000, reps=5):
    """The perceptron forward alone (ten outputs, one row per node of the reacting
    workload): the warp-level BF16 MMA path against the tcgen05 path, host wall time per
    call (each synchronises), best of reps; tensor FLOPs = the two BF16 layers as executed
    (K padded to 16 in layer 1) over the measured dense BF16 peak."""
    import torch
    import paper_2511_17551_gb300 as dg
    rng = np.random.default_rng(5)
    P = torch.from_numpy((0.3 * rng.normal(size=dg.dg_mlp_nparams(10))).astype(np.float32)).cuda()
    X = torch.from_numpy(rng.normal(size=(n, 7)).astype(np.float32)).cuda()
    y = torch.empty((n, 10), dtype=torch.float32, device="cuda")
    flops_row = 2 * (16 * 64 + 64 * 64)
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops") \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
    out = {"rows": n, "n_out": 10, "tensor_flops_per_row": flops_row, "bf16_peak_tflops": peak}
    for name, tc in (("warp_mma_sync", 1), ("tcgen05", 2)):
        dg.dg_mlp_forward(P, X, y, tensor_cores=tc)
        best = 1e9
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dg.dg_mlp_forward(P, X, y, tensor_cores=tc)
            best = min(best, time.perf_counter() - t0)
        out[name] = {"ms": best * 1e3, "tensor_tflops": flops_row * n / best / 1e12,
                     "frac_of_bf16_peak": flops_row * n / best / 1e12 / peak}
    return out


# FP64 flops per node of the FP64-pipe-bound kernels of the mixture workloads (2 DFMA +
# DMUL + DADD thread instructions over the nodes, one ncu capture each: mixture 16^3 and
# reacting 24 x 24 x 8, N = 4, mixed form).  The temperature solve's count depends on the
# Newton iterations its states need (1 to 2 from the cached temperature there).
THERMO_FP64_FLOPS_PER_NODE = 119.0
CHEM_FP64_FLOPS_PER_NODE = 1714.0


def _fp64_roofline(kernel, flops_per_node, nodes, ms_per_launch, fp64_peak):
    achieved = flops_per_node * nodes / (ms_per_launch * 1e-3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "flops_per_node": flops_per_node, "ms_per_launch": ms_per_launch,
            "peak_source": "FP64 FMA chains measured here (dg_peak_flops); the FP64 pipe binds"}


def _timed_run(dg, torch, s, w0, n, cfl):
    """n CK45 steps from the primitive state w0 with per-kernel device timing: (state,
    wall ms per step, {kind: (ms, launches)}); the state is None when the run stopped on a
    latched device error (message in the wall slot)."""
    s.set_primitive(w0)
    dg.dg_profile(s.ctx, 1)
    dg.dg_profile_read(s.ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        s.step(n, cfl)
    except dg.DgError as e:
        dg.dg_profile(s.ctx, 0)
        return None, str(e), {}
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3 / n
    prof = dg.dg_profile_read(s.ctx)
    dg.dg_profile(s.ctx, 0)
    return s.get_state()[0], wall, prof


def _per_step(prof, n):
    return {k: round(v[0] / n, 4) for k, v in prof.items() if v[1]}


def run_mixture(args, stream_ptr, world, fp64_peak):
    """Five-species frozen mixture on the 24^3-element cylinder O-grid, N = 4 (Mach 5 nominal),
    args.mix_steps CK45 steps from the same state in three forms: the FP64 plain form, the
    mixed form with the plain Newton temperature solve, and the mixed form with the learned
    temperature (trained here on states of the plain solver's own run); per-field relative
    L2 of each mixed run's end state and the temperature's max relative difference against
    the FP64 form's.  Also the learned temperature's gain over a cold and a converged-cache
    Newton solve (thermo kernel time alone) and the limiter's cost."""
    import torch
    import paper_2511_17551_gb300 as dg
    from paper_2511_17551_gb300 import surrogate as S
    N, nr = 4, args.mix_elements
    xi, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face = W.ogrid_mesh(xi, nr, nr, nr)
    # potential flow past the cylinder as the start (tangent at the wall), free stream at
    # the far field; subcell-FV blending (alpha <= 0.5) captures the bow shock that forms
    w0 = W.mixture_primitive(xyz, rho=0.1, vel=(2000.0, 0.0, 0.0), T=300.0, seed=7, cylinder=0.5)
    fs = W.mixture_primitive(xyz[:1], rho=0.1, vel=(2000.0, 0.0, 0.0), T=300.0, seed=7)[0, :, 0]
    K, npn = xyz.shape[0], (N + 1) ** 3
    dof = K * npn * 9  # 5 species densities, 3 momenta, energy
    steps = max(2, args.mix_steps)
    sp = W.species_table()
    cfl = 0.3

    def make(precision, positivity_eps=0.0):
        s = dg.Solver(3, N, xyz, nbr, face, n_species=5, species=sp, volume_flux=dg.DG_VF_DUCROS,
                      surface_flux=dg.DG_SF_LLF, bc_kind=[1, 2, 3], bc_prim=np.stack([fs] * 3),
                      alpha_max=0.5, precision=precision, stream=stream_ptr, positivity_eps=positivity_eps)
        s.set_primitive(w0)
        return s

    def form(u, wall, prof, u_ref=None, T=None, T_ref=None):
        d = {"value": world * dof * 5 / (wall * 1e-3), "ms_per_step": wall,
             "device_ms_per_step_by_kernel": _per_step(prof, steps)}
        if u_ref is not None:
            d["l2_vs_fp64_form"] = field_errors(u, u_ref, nsp=5)
        if T_ref is not None:
            d["T_max_rel_vs_fp64_form"] = float(np.abs(T / T_ref - 1).max())
        return d

    out = {"workload": "mixture_5sp_ogrid_%d^3_N4" % nr, "elements": K, "dof": dof, "steps": steps,
           "cfl": cfl, "norm": "relative L2 per conserved field (R19) of the end state after `steps` "
           "CK45 steps from the same state, against the FP64 plain form (itself checked against the "
           "oracle to 1e-12 per right-hand side by the test suite)"}
    s64 = make(dg.DG_FP64)
    u64, wall, prof = _timed_run(dg, torch, s64, w0, steps, cfl)
    T64 = dg.dg_get_temperature(s64.ctx, (K, npn))
    out["fp64_newton"] = form(u64, wall, prof)
    s64.close()
    s = make(dg.DG_MIXED)
    um, wall, prof = _timed_run(dg, torch, s, w0, steps, cfl)
    Tm = dg.dg_get_temperature(s.ctx, (K, npn))
    out["mixed_newton"] = form(um, wall, prof, u64, Tm, T64)
    th_ms = prof["thermo"][0] / max(1, prof["thermo"][1])
    out["mixed_newton"]["thermo_ms_per_launch"] = th_ms
    out["mixed_newton"]["rhs_ms_per_launch"] = prof["rhs"][0] / max(1, prof["rhs"][1])
    out["roofline"] = _fp64_roofline("thermo_update_kernel<float> (mixed form, the block's dominant kernel)",
                                     THERMO_FP64_FLOPS_PER_NODE, K * npn, th_ms, fp64_peak)
    # the same with the mixture positivity limiter after every stage (partial densities
    # >= 1e-9 kg/m^3, T >= 200 K): its screening pass and any limiting it does
    sl = make(dg.DG_MIXED, positivity_eps=1e-9)
    ul, wl, pl = _timed_run(dg, torch, sl, w0, steps, cfl)
    out["mixed_newton_limiter"] = {"ms_per_step": wl, "limited_element_stages": dg.dg_limiter_stats(sl.ctx),
                                   "device_ms_per_step_by_kernel": _per_step(pl, steps)}
    sl.close()
    # training data from the plain solver's own run, then the surrogate
    t0 = time.perf_counter()
    s.set_primitive(w0)
    X, T = S.collect(s.ctx, args.train_samples, 10, 2, cfl=cfl)
    params, stats, hist = S.train(X, T, epochs=args.train_epochs, batch=4096, lr=2e-3, lr_final=1e-4)
    out["training"] = {"samples": int(X.shape[0]), "epochs": args.train_epochs,
                       "val_mse_first_last": [hist[0][2], hist[-1][2]],
                       "seconds": time.perf_counter() - t0}
    # gain on the thermo kernel alone: cold Newton, converged-cache Newton, surrogate
    Tshape = (K, npn)
    s.set_primitive(w0)
    dg.dg_profile(s.ctx, 1)
    dg.dg_profile_read(s.ctx)
    s.set_primitive(w0)
    T_cold = dg.dg_get_temperature(s.ctx, Tshape)
    cold = dg.dg_profile_read(s.ctx)["thermo"][0]
    dg.dg_get_temperature(s.ctx, Tshape)
    warm = dg.dg_profile_read(s.ctx)["thermo"][0]
    dg.dg_set_surrogate(s.ctx, params, stats)
    dg.dg_surrogate_stats(s.ctx)
    T_mlp = dg.dg_get_temperature(s.ctx, Tshape)
    mlp = dg.dg_profile_read(s.ctx)["thermo"][0]
    acc, fb = dg.dg_surrogate_stats(s.ctx)
    dg.dg_profile(s.ctx, 0)
    out["thermo_gain"] = {"cold_newton_ms": cold, "converged_cache_newton_ms": warm,
                          "surrogate_ms": mlp, "gain_vs_converged_cache": warm / mlp,
                          "accepted": acc, "fallback": fb,
                          "max_rel_T_diff_vs_newton": float(np.abs(T_mlp / T_cold - 1).max()),
                          "verdict": "the learned temperature costs more than the plain FP32 Newton "
                                     "iteration it replaces (1-2 iterations from the cached T)"}
    dg.dg_surrogate_stats(s.ctx)
    ul, wall, prof = _timed_run(dg, torch, s, w0, steps, cfl)
    Tl = dg.dg_get_temperature(s.ctx, (K, npn))
    acc, fb = dg.dg_surrogate_stats(s.ctx)
    out["mixed_surrogate"] = form(ul, wall, prof, u64, Tl, T64)
    out["mixed_surrogate"]["thermo_ms_per_launch"] = prof["thermo"][0] / max(1, prof["thermo"][1])
    out["mixed_surrogate"]["accept_frac"] = acc / max(1, acc + fb)
    s.close()
    out["_surrogate"] = (params, stats)
    return out


def run_reacting(args, stream_ptr, world, fp64_peak):
    """Five-species reacting mixture (17 reactions, FP64 finite-rate source with point-implicit
    scaling) on a 48 x 48 x 16-element cylinder O-grid, N = 4, with a 3000 K layer round the
    body: args.react_steps CK45 steps from the same state in the FP64 plain form, the mixed
    form with the plain source, and the mixed form with the learned source (trained here on
    states of the plain run) at the default acceptance tolerance 0.05 and at 0.01, and with
    the plain correction (refresh every 1 or 2 steps);
    throughput, per-kernel device time, and per-field relative L2 of each mixed run's end
    state against the FP64 form's."""
    import torch
    import paper_2511_17551_gb300 as dg
    from paper_2511_17551_gb300 import surrogate as S
    N = 4
    nr, nth, nz = args.react_elements, args.react_elements, max(2, args.react_elements // 3)
    xi, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face = W.ogrid_mesh(xi, nr, nth, nz)
    sp, R = W.species_table(), W.reaction_table()
    u_inf = (2400.0, 0.0, 0.0)
    w0 = W.mixture_primitive(xyz, rho=0.1, vel=u_inf, T=300.0, seed=7, cylinder=0.5,
                             hot=(1.2, 3000.0))
    fs = W.mixture_primitive(xyz[:1], rho=0.1, vel=u_inf, T=300.0, seed=7)[0, :, 0]
    K, npn = xyz.shape[0], (N + 1) ** 3
    dof = K * npn * 9  # 5 species densities, 3 momenta, energy
    cfl = 0.05
    n = max(1, args.react_steps)
    out = {"workload": "reacting_5sp_17r_ogrid_%dx%dx%d_N4" % (nr, nth, nz), "elements": K,
           "dof": dof, "cfl": cfl, "steps": n,
           "norm": "relative L2 per conserved field (R19) of the end state after `steps` CK45 steps "
                   "from the same state, against the FP64 plain form (itself checked against the "
                   "oracle to 1e-12 per right-hand side by the test suite)"}

    def make(prec):
        s = dg.Solver(3, N, xyz, nbr, face, n_species=5, species=sp, volume_flux=dg.DG_VF_DUCROS,
                      surface_flux=dg.DG_SF_LLF, bc_kind=[1, 2, 3], bc_prim=np.stack([fs] * 3),
                      alpha_max=0.5, precision=prec, reactions=R, stream=stream_ptr)
        s.set_primitive(w0)
        return s

    def form(u, wall, prof, u_ref=None):
        if u is None:
            return {"error": wall}
        chem_ms = prof["chem"][0] / max(1, prof["chem"][1])
        d = {"value": world * dof * 5 / (wall * 1e-3), "unit": "DOF*RHS/s", "ms_per_step": wall,
             "chem_ms_per_launch": chem_ms, "chem_ns_per_node": chem_ms * 1e6 / (K * npn),
             "device_ms_per_step_by_kernel": _per_step(prof, n)}
        if u_ref is not None:
            d["l2_vs_fp64_form"] = field_errors(u, u_ref, nsp=5)
        return d

    s64 = make(dg.DG_FP64)
    u64, wall, prof = _timed_run(dg, torch, s64, w0, n, cfl)
    out["fp64"] = form(u64, wall, prof)
    s64.close()
    s = make(dg.DG_MIXED)
    um, wall, prof = _timed_run(dg, torch, s, w0, n, cfl)
    out["mixed"] = form(um, wall, prof, u64)
    if um is not None:
        out["roofline"] = _fp64_roofline("chem_kernel<float> (mixed form, the block's dominant kernel)",
                                         CHEM_FP64_FLOPS_PER_NODE, K * npn, out["mixed"]["chem_ms_per_launch"],
                                         fp64_peak)
    # learned source: data from the plain run's own states (8 snapshots spread over the
    # run's length), training, the same steps again
    t0 = time.perf_counter()
    s.set_primitive(w0)
    X, Y = S.collect_source(s.ctx, args.train_samples, 8, max(1, n // 8), cfl=cfl)
    params, stats, hist = S.train_source(X, Y, epochs=args.train_epochs, batch=4096, lr=3e-3, lr_final=1e-4)
    train_s = time.perf_counter() - t0
    out["training"] = {"samples": int(X.shape[0]), "epochs": args.train_epochs,
                       "val_mse_first_last": [hist[0][2], hist[-1][2]], "seconds": train_s}
    # the learned source alone at two tolerances, and with the plain correction (a refresh
    # at the first stage of every k-th step, the refresh's full check at the same tolerance)
    for key, tol, k in (("mixed_learned_source", 0.05, 0), ("mixed_learned_source_tol0.01", 0.01, 0),
                        ("mixed_corrected_source_tol0.002_k1", 0.002, 1),
                        ("mixed_corrected_source_tol0.002_k2", 0.002, 2),
                        ("mixed_corrected_source_tol0.01_k1", 0.01, 1),
                        ("mixed_corrected_source_tol0.01_k2", 0.01, 2)):
        st = stats.copy()
        st[50] = st[51] = tol
        dg.dg_set_surrogate(s.ctx, params, st, which=dg.DG_SURROGATE_SOURCE)
        dg.dg_set_source_refresh(s.ctx, k)
        dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        ul, wall, prof = _timed_run(dg, torch, s, w0, n, cfl)
        acc, fb = dg.dg_surrogate_stats(s.ctx, dg.DG_SURROGATE_SOURCE)
        d = form(ul, wall, prof, u64)
        d["tolerance"] = tol
        d["refresh_period_steps"] = k
        d["accepted_node_fraction"] = acc / max(1, acc + fb)
        if k:
            d["refresh_evaluations_per_step"] = 1.0 / k
        out[key] = d
        if ul is None:
            s.close()
            s = make(dg.DG_MIXED)
    s.close()
    return out


def run_other_shapes(args, stream_ptr, world):
    """The other full-size shapes: NS Taylor-Green 16^3 at N = 7 (same DOF as the headline)
    and the 2D Mach-3 square cylinder (512 x 256 quads less the body, N = 3, shock capturing
    with alpha <= 0.5), both forms; DOF*RHS-evals/s and per-kernel device time per step."""
    import torch
    import paper_2511_17551_gb300 as dg
    out = {}

    def timed(s, n, cfl):
        s.step(2, cfl)
        dg.dg_profile(s.ctx, 1)
        dg.dg_profile_read(s.ctx)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(n, cfl)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        prof = dg.dg_profile_read(s.ctx)
        dg.dg_profile(s.ctx, 0)
        return wall, {k: round(v[0] / n, 4) for k, v in prof.items() if v[1]}

    # NS TGV 16^3, N = 7
    cfg = CONFIGS["tgv_ns_16^3_N7"]
    xi, _ = dg.dg_lgl_nodes(cfg["N"])
    xyz, nbr, face, w0 = build_workload(cfg, xi)
    dof = xyz.shape[0] * (cfg["N"] + 1) ** 3 * 5
    blk = {"workload": "tgv_ns_16^3_N7", "dof": dof}
    for name, prec, n in (("mixed", dg.DG_MIXED, 50), ("fp64", dg.DG_FP64, 3)):
        s = dg.Solver(3, cfg["N"], xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=cfg["mu"],
                      Pr=0.72, precision=prec, stream=stream_ptr, p_ref=1.0 / (1.4 * 0.01))
        s.set_primitive(w0)
        wall, per = timed(s, n, 0.5)
        s.close()
        blk[name] = {"value": world * dof * 5 * n / wall, "ms_per_step": wall * 1e3 / n, "steps": n,
                     "device_ms_per_step_by_kernel": per}
    out["tgv_ns_16^3_N7"] = blk
    # the split-form volume fluxes and the interface fluxes on the bench workload (TGV
    # Navier-Stokes 32^3, N = 3, mixed form): ranocha_llf is the production pair of the
    # headline number, the other *_llf pairs run their compile-time kernels, the rest the
    # runtime-choice kernel
    cfg = CONFIGS["tgv_ns_32^3_N3"]
    xi, _ = dg.dg_lgl_nodes(cfg["N"])
    xyz, nbr, face, w0 = build_workload(cfg, xi)
    dof = xyz.shape[0] * (cfg["N"] + 1) ** 3 * 5
    blk = {"workload": "tgv_ns_32^3_N3", "dof": dof, "form": "mixed", "steps": 20}
    for name, vf, sf in (("ranocha_llf", dg.DG_VF_RANOCHA, dg.DG_SF_LLF),
                         ("kennedy_gruber_llf", dg.DG_VF_KG, dg.DG_SF_LLF),
                         ("pirozzoli_llf", dg.DG_VF_PIROZZOLI, dg.DG_SF_LLF),
                         ("morinishi_llf", dg.DG_VF_MORINISHI, dg.DG_SF_LLF),
                         ("ducros_llf", dg.DG_VF_DUCROS, dg.DG_SF_LLF),
                         ("standard_dg_llf", dg.DG_VF_CENTRAL, dg.DG_SF_LLF),
                         ("kennedy_gruber_hll", dg.DG_VF_KG, dg.DG_SF_HLL),
                         ("pirozzoli_hllc", dg.DG_VF_PIROZZOLI, dg.DG_SF_HLLC),
                         ("ducros_ec", dg.DG_VF_DUCROS, dg.DG_SF_EC)):
        s = dg.Solver(3, cfg["N"], xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=cfg["mu"],
                      Pr=0.72, precision=dg.DG_MIXED, stream=stream_ptr, p_ref=1.0 / (1.4 * 0.01),
                      volume_flux=vf, surface_flux=sf)
        s.set_primitive(w0)
        wall, per = timed(s, 20, 0.5)
        s.close()
        blk[name] = {"value": world * dof * 5 * 20 / wall, "ms_per_step": wall * 1e3 / 20,
                     "device_ms_per_step_by_kernel": per}
    out["split_forms_tgv_ns_32^3_N3"] = blk
    # wall-bounded channel, 64 x 16 x 32 elements, N = 3: periodic in x and z, a no-slip
    # adiabatic wall at y = 0 and an isothermal wall at y = 1 (BR1 boundary values, boundary
    # viscous fluxes and the boundary lifting kernel), Mach-0.1 shear flow, Re 1600
    xi, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face = W.box_mesh((64, 16, 32), xi, (0.0, 0.0, 0.0), (4.0, 1.0, 2.0),
                                periodic=(True, False, True), bc_ids=[9, 9, 0, 1, 9, 9])
    p0 = 1.0 / (1.4 * 0.01)
    w0 = W.channel_primitive(xyz, p0)
    dof = xyz.shape[0] * 64 * 5
    blk = {"workload": "channel_walls_64x16x32_N3", "dof": dof, "walls": "no-slip adiabatic / isothermal",
           "Re": 1600}
    for name, prec, n in (("mixed", dg.DG_MIXED, 20), ("fp64", dg.DG_FP64, 3)):
        s = dg.Solver(3, 3, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=1.0 / 1600.0,
                      Pr=0.72, precision=prec, stream=stream_ptr, p_ref=p0,
                      bc_kind=[dg.DG_BC_NOSLIP_ADIABATIC, dg.DG_BC_ISOTHERMAL],
                      bc_prim=np.array([[1.0, 0.0, 0.0, 0.0, p0]] * 2))
        s.set_primitive(w0)
        wall, per = timed(s, n, 0.5)
        s.close()
        blk[name] = {"value": world * dof * 5 * n / wall, "ms_per_step": wall * 1e3 / n, "steps": n,
                     "device_ms_per_step_by_kernel": per}
    out["channel_walls_64x16x32_N3"] = blk
    # supersonic TGV 32^3, N = 7: Sutherland's law, pressure-indicator blending, positivity
    n_el, N = 32, 7
    xi, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face = W.box_mesh((n_el,) * 3, xi, (-np.pi,) * 3, (np.pi,) * 3, periodic=True)
    w0 = W.supersonic_tgv_primitive(xyz)
    dof = xyz.shape[0] * (N + 1) ** 3 * 5
    phys = W.supersonic_tgv_physics()
    blk = {"workload": "supersonic_tgv_32^3_N7", "dof": dof, "mach": 1.25, "Re": 1600,
           "alpha_max": 0.5, "positivity_eps": 1e-8, "cfl": 0.4}
    for name, prec, n in (("mixed", dg.DG_MIXED, 20), ("fp64", dg.DG_FP64, 3)):
        s = dg.Solver(3, N, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, alpha_max=0.5,
                      precision=prec, stream=stream_ptr, positivity_eps=1e-8, **phys)
        s.set_primitive(w0)
        try:
            wall, per = timed(s, n, 0.4)
            blk[name] = {"value": world * dof * 5 * n / wall, "ms_per_step": wall * 1e3 / n, "steps": n,
                         "blended_elements": int((dg.dg_get_alpha(s.ctx, s.K) > 0).sum()),
                         "device_ms_per_step_by_kernel": per}
        except dg.DgError as e:
            blk[name] = {"error": str(e)}
        s.close()
    out["supersonic_tgv_32^3_N7"] = blk
    # 2D Mach-3 square cylinder
    xi, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face = W.square_cylinder_mesh(xi)
    gamma, mach = 1.4, 3.0
    fs = np.array([1.0, 1.0, 0.0, 1.0 / (gamma * mach * mach)])
    w0 = W.freestream_primitive(xyz.shape[0], 16, fs)
    dof = xyz.shape[0] * 16 * 4
    blk = {"workload": "square_cylinder_mach3_512x256_N3", "elements": xyz.shape[0], "dof": dof,
           "alpha_max": 0.5, "cfl": 0.3, "positivity_eps": 1e-10}
    for name, prec, n in (("mixed", dg.DG_MIXED, 40), ("fp64", dg.DG_FP64, 10)):
        s = dg.Solver(2, 3, xyz, nbr, face, bc_kind=[1, 2, 3], bc_prim=np.stack([fs] * 3),
                      alpha_max=0.5, precision=prec, stream=stream_ptr, positivity_eps=1e-10)
        s.set_primitive(w0)
        try:
            wall, per = timed(s, n, 0.3)
            blk[name] = {"value": world * dof * 5 * n / wall, "ms_per_step": wall * 1e3 / n, "steps": n,
                         "blended_elements": int((dg.dg_get_alpha(s.ctx, s.K) > 0).sum()),
                         "limited_element_stages": dg.dg_limiter_stats(s.ctx),
                         "device_ms_per_step_by_kernel": per}
        except dg.DgError as e:
            blk[name] = {"error": str(e)}
        s.close()
    out["square_cylinder"] = blk
    return out


def cpu_baseline(cfg, budget_s):
    """The oracle as it stands, FP64, all host cores (OpenMP over elements): CK45 steps of
    the workload at a fixed step (the oracle's CFL-0.5 step of the initial state) for about
    budget_s seconds.  Also returns, for the parity report, the oracle's right-hand side of
    the initial state and its state after those steps."""
    import oracle
    N = cfg["N"]
    xo, _ = oracle.lgl(N)
    xyz, nbr, face, w0 = build_workload(cfg, xo)
    o = oracle.Oracle(3, N, xyz, nbr, face, equations=1 if cfg["mu"] > 0 else 0, mu=cfg["mu"],
                      Pr=0.72)
    u = o.prim_to_cons(w0)
    r0 = o.rhs(u)
    # the oracle's own rounding floor for this right-hand side: its change when every state
    # value moves by one unit in the last place (seeded signs), before the timed steps
    sgn = np.random.default_rng(5).choice([-1.0, 1.0], size=u.shape)
    floor = field_errors(o.rhs(u * (1.0 + np.finfo(np.float64).eps * sgn)), r0)
    # and to one FP32 unit of every state value: the floor of any right-hand side that is
    # computed from an FP32 state
    floor32 = field_errors(o.rhs(u * (1.0 + 2.0 ** -24 * sgn)), r0)
    u_init = u.copy()
    dt_step = o.max_dt(u, 0.5)
    dof = u.size
    n, t0 = 0, time.perf_counter()
    while True:
        u, _ = o.step_rk(u, 1, dt_fixed=dt_step)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    wall = time.perf_counter() - t0
    cores = oracle.set_threads(0)
    info = {"value": dof * 5 * n / wall, "unit": "DOF*RHS/s", "cores": cores, "kind": "oracle",
            "sample": "%d CK45 steps (%d right-hand sides) of the full %d-element workload in %.1f s" % (
                n, 5 * n, xyz.shape[0], wall), "cpu_model": _cpu_model()}
    # one thread: right-hand sides of the same workload for a bounded time
    oracle.set_threads(1)
    u1 = o.prim_to_cons(w0)
    n1, t1 = 0, time.perf_counter()
    while True:
        o.rhs(u1)
        n1 += 1
        if time.perf_counter() - t1 > max(2.0, budget_s / 3):
            break
    w1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    info["single_thread"] = {"value": dof * n1 / w1, "unit": "DOF*RHS/s", "cores": 1,
                             "sample": "%d right-hand sides of the full workload in %.1f s" % (n1, w1)}
    return info, r0, u, n, dt_step, (floor, floor32, u_init)


def _cpu_model():
    """Host CPU model (lscpu's model name, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def mixture_T_vs_oracle(args, surrogate):
    """The five-species mixture's initial state (same seeded primitive field): the oracle's
    Newton temperature against the GPU's FP64 Newton, mixed-form Newton and learned
    temperature (max relative difference over the nodes)."""
    import oracle
    import paper_2511_17551_gb300 as dg
    N, nr = 4, args.mix_elements
    res = {}
    xo, _ = oracle.lgl(N)
    xyz_o, nbr, face = W.ogrid_mesh(xo, nr, nr, nr)
    w_o = W.mixture_primitive(xyz_o, rho=0.1, vel=(2000.0, 0.0, 0.0), T=300.0, seed=7, cylinder=0.5)
    o = oracle.Oracle(3, N, xyz_o, nbr, face, n_species=5, species=W.species_table(), volume_flux=1)
    T_o = o.temperature(o.prim_to_cons(w_o))
    xi, _ = dg.dg_lgl_nodes(N)
    xyz, nbr, face = W.ogrid_mesh(xi, nr, nr, nr)
    w0 = W.mixture_primitive(xyz, rho=0.1, vel=(2000.0, 0.0, 0.0), T=300.0, seed=7, cylinder=0.5)
    fs = w0[0, :, 0]
    for name, prec, use in (("fp64_newton", dg.DG_FP64, False), ("mixed_newton", dg.DG_MIXED, False),
                            ("mixed_surrogate", dg.DG_MIXED, True)):
        if use and surrogate is None:
            continue
        s = dg.Solver(3, N, xyz, nbr, face, n_species=5, species=W.species_table(), volume_flux=1,
                      bc_kind=[1, 2, 3], bc_prim=np.stack([fs] * 3), precision=prec)
        s.set_primitive(w0)
        if use:
            dg.dg_set_surrogate(s.ctx, surrogate[0], surrogate[1])
        T = dg.dg_get_temperature(s.ctx, (s.K, s.np))
        res[name] = float(np.abs(T / T_o - 1).max())
        s.close()
    return res


def field_errors(a, ref, dim=3, nsp=1):
    """Relative L2 error per conserved field (species densities, momenta, energy; momentum
    components over the norm of the whole momentum block)."""
    mom = np.linalg.norm(ref[:, nsp:nsp + dim])
    return [float(np.linalg.norm(a[:, v] - ref[:, v]) /
                  (mom if nsp <= v < nsp + dim else np.linalg.norm(ref[:, v]))) for v in range(a.shape[1])]


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    cfg = CONFIGS[args.config]
    N = cfg["N"]
    xo, _ = oracle.lgl(N)
    # bounded sample: the same TGV at 8^3 elements (same N, mesh warp and physics)
    n_el = min(cfg["n_el"], 8)
    xyz, nbr, face = W.box_mesh((n_el,) * 3, xo, (-np.pi,) * 3, (np.pi,) * 3, periodic=True,
                                warp=cfg["warp"])
    o = oracle.Oracle(3, N, xyz, nbr, face, equations=1 if cfg["mu"] > 0 else 0, mu=cfg["mu"],
                      Pr=0.72)
    u = o.prim_to_cons(W.tgv_primitive(xyz))
    dof = u.size
    u, _ = o.step_rk(u, args.warmup)
    t0 = time.perf_counter()
    u, _ = o.step_rk(u, args.steps)
    dt = time.perf_counter() - t0
    value = dof * 5 * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    sample = "%d^3-element cut of %s, %d CK45 steps" % (n_el, args.config, args.steps)
    print(json.dumps({
        "impl": "reference", "metric": "DOF*RHS-evals/s (FP32+FP64-reductions form; FP64 form beside it)",
        "value": value, "unit": "DOF*RHS/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "elements_sampled": n_el ** 3, "N": N},
        "cpu_baseline": {"value": value, "unit": "DOF*RHS/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "DOF*RHS/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def run_profile_case(name):
    """Small cases for ncu section captures (2 RK steps, then exit): 'fp64rhs' (NS TGV 16^3,
    N = 3, FP64 form), 'mixture' (5-species O-grid 16^3, N = 4, mixed), 'reacting'
    (reacting O-grid 24 x 24 x 8, N = 4, mixed); 'mlp' (the tcgen05 perceptron forward,
    1 M rows, three calls)."""
    import torch
    import paper_2511_17551_gb300 as dg
    if name == "mlp":
        # the perceptron forward on the tcgen05 path, ten outputs, 1 M rows (3 calls)
        rng = np.random.default_rng(5)
        P = torch.from_numpy((0.3 * rng.normal(size=dg.dg_mlp_nparams(10))).astype(np.float32)).cuda()
        X = torch.from_numpy(rng.normal(size=(1_000_000, 7)).astype(np.float32)).cuda()
        y = torch.empty((1_000_000, 10), dtype=torch.float32, device="cuda")
        for _ in range(3):
            dg.dg_mlp_forward(P, X, y, tensor_cores=2)
        torch.cuda.synchronize()
        return
    if name == "fp64rhs":
        N = 3
        xi, _ = dg.dg_lgl_nodes(N)
        xyz, nbr, face = W.box_mesh((16,) * 3, xi, (-np.pi,) * 3, (np.pi,) * 3, periodic=True, warp=0.1)
        s = dg.Solver(3, N, xyz, nbr, face, equations=dg.DG_NAVIER_STOKES, mu=1.0 / 1600.0, Pr=0.72,
                      precision=dg.DG_FP64, p_ref=1.0 / (1.4 * 0.01))
        s.set_primitive(W.tgv_primitive(xyz))
        s.step(2, 0.5)
    else:
        N = 4
        xi, _ = dg.dg_lgl_nodes(N)
        react = name == "reacting"
        xyz, nbr, face = W.ogrid_mesh(xi, *((24, 24, 8) if react else (16, 16, 16)))
        vel = (2400.0 if react else 2000.0, 0.0, 0.0)
        hot = (1.2, 3000.0) if react else None
        w0 = W.mixture_primitive(xyz, rho=0.1, vel=vel, T=300.0, seed=7, cylinder=0.5, hot=hot)
        fs = W.mixture_primitive(xyz[:1], rho=0.1, vel=vel, T=300.0, seed=7)[0, :, 0]
        s = dg.Solver(3, N, xyz, nbr, face, n_species=5, species=W.species_table(),
                      volume_flux=dg.DG_VF_DUCROS, surface_flux=dg.DG_SF_LLF, bc_kind=[1, 2, 3],
                      bc_prim=np.stack([fs] * 3), alpha_max=0.5, precision=dg.DG_MIXED,
                      reactions=W.reaction_table() if react else None)
        s.set_primitive(w0)
        s.step(2, 0.05 if react else 0.3)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "nodes": s.K * s.np}))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="tgv_ns_32^3_N3", choices=sorted(CONFIGS))
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixture", action="store_true")
    ap.add_argument("--mix-elements", type=int, default=24, help="O-grid elements per direction")
    ap.add_argument("--mix-steps", type=int, default=100)
    ap.add_argument("--train-samples", type=int, default=1000000)
    ap.add_argument("--train-epochs", type=int, default=60, help="epochs of each surrogate's training "
                    "(Adam, step size decaying by a cosine to 1e-4)")
    ap.add_argument("--no-reacting", action="store_true")
    ap.add_argument("--no-other-shapes", action="store_true",
                    help="skip the 16^3 N=7 Taylor-Green and the square-cylinder blocks")
    ap.add_argument("--react-elements", type=int, default=48, help="O-grid radial/angular elements")
    ap.add_argument("--react-steps", type=int, default=100,
                    help="CK45 steps of each reacting run (the reacting configuration asks 500)")
    ap.add_argument("--profile-case", choices=["fp64rhs", "mixture", "reacting", "mlp"],
                    help="run one small case for an ncu capture and exit")
    args = ap.parse_args()
    rank, world, local_rank = _env_rank()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
