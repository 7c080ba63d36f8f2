#!/usr/bin/env python
"""Benchmark: BiCGSTAB-GMG stage solve to true relative residual 1e-10.

Workload (one step = one solve from x0 = 0): the 257^3-vertex box with a
lognormal permeability field (seed 2) and six low-K lenses, stage matrix
A = M/h - J at h = 10 s assembled at the initial state, right-hand side F(u0);
FP64 BiCGSTAB preconditioned by one FP32 V(2,2)-cycle (7 levels, 8-colour
block Gauss-Seidel).  The metric is DoF/s = 2 * vertices / solve time, with the
multigrid set-up excluded (reported separately, as are the assembly and the
all-FP64 and FP16-storage variants of the same solve).

Inputs stay resident in HBM; the FP64 Jacobian alone (14.7 GB) is far larger
than L2, so nothing is flushed between steps.  `--impl reference` times the
CPU oracle (single thread, FP64) on a bounded sample of the same recipe.
Under torchrun (N > 1) every rank solves its own replica (the path is one
coupled problem, so ranks do not shard it); value = total DoF/s.
"""
import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


class _Skip(Exception):
    """A bench block switched off on the command line."""


METRIC = "BiCGSTAB-GMG DoF/s to rel.res 1e-10, FP32-GMG vs FP64, % of HBM peak"
RTOL = 1e-10
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per updated vertex
# of a full fine-level FP32 GS launch, by launch form (one launch per colour
# pair, the default, or per colour with RF_GS_PAIRS=0) and vertices per axis of
# this workload's recipe: ncu captures of the launches of the second fine
# sweep in the solve's own launch sequence (caches not flushed, so a launch
# finds in L2 what its predecessors left); the algorithmic count is 456 B.
GS_TRAFFIC_PER_VERTEX = {"pair": {257: 496.2}, "colour": {257: 516.6}}
GS_ALGO_PER_VERTEX = 456.0
# FP64 floating-point operations per vertex of one outer operator application
# (k_bicg_v / k_bicg_t): 27 blocks x 4 FMA (216 flop), the shift*M diagonal
# (4 flop) and the fused inner products (<rh, v>: 4 flop; <t, s>, <t, t>: 8
# flop), averaged over the two applications of an iteration.
SPMV64_FLOP_PER_VERTEX = 216.0 + 4.0 + 6.0
# FP64 instructions (DADD + DMUL + DFMA) per vertex of one K1 assembly with the
# Jacobian, counted by ncu (smsp__sass_thread_inst_executed_op_d{add,mul,fma})
# over the 8 colour launches of one assembly of this recipe at 129^3; K1 is
# FP64-issue-bound, so its roofline is that instruction rate against the FMA
# issue rate rf_fp64_fma_rate measures.
K1_FP64_INST_PER_VERTEX = 4154.0


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nvert", type=int, default=257)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--smoother", default="gs8", choices=["gs8", "jacobi"])
    ap.add_argument("--outer", default="fp64", choices=["fp64", "df32"],
                    help="arithmetic of the operator applications inside the iteration")
    ap.add_argument("--variants", default="fp64,fp16,fp32+df32",
                    help="extra solve variants to time: precision[+outer], comma separated ('none': no variants)")
    ap.add_argument("--sample-nvert", type=int, default=129, help="oracle sample size (vertices per axis)")
    ap.add_argument("--ensemble", type=int, default=1, help="also time the 64-realisation ensemble (1/0)")
    ap.add_argument("--limex", type=int, default=1, help="also time one 65^3 LIMEX step and its schedules (1/0)")
    ap.add_argument("--infiltration-nvert", type=int, default=385,
                    help="also run adaptive LIMEX on the DNAPL-infiltration recipe at this size (0: skip)")
    ap.add_argument("--infiltration-steps", type=int, default=3,
                    help="accepted steps of the infiltration run (the workload's 20 take ~3 minutes)")
    ap.add_argument("--case4-days", type=float, default=0.0,
                    help="also run the layered Case-4 analogue for this many days with implicit Euler (1-day steps) "
                         "and adaptive LIMEX (0 = off)")
    ap.add_argument("--case4-nvert", default="257x129", help="Case-4 analogue vertices (x by y)")
    ap.add_argument("--autotune", type=int, default=0,
                    help="time block sizes of the level kernels during the set-up (1/0)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm=d.get("hbm_gbs", 6800.0), src="measured")
    return dict(hbm=6800.0, src="fallback")


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        # raw samples: RF_CLOCKS_CSV names the file (default: a temporary one)
        self.path = os.environ.get("RF_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(), "rf_clocks_bench.csv")
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        self.p = None
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [t.strip() for t in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx.append(float(c[2]))
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if c[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle baseline
def host_cores():
    return len(os.sched_getaffinity(0))


class OracleSample:
    """The CPU oracle (as it stands) on the same recipe at a bounded size: the
    system is assembled and the multigrid set up once; solve(threads) times one
    BiCGSTAB-GMG solve from x0 = 0 to 1e-10 with that many OpenMP threads
    (results are bitwise the same for any count).  Returns (DoF/s, seconds,
    iterations)."""

    def __init__(self, nvert, smoother):
        import oracle as O
        from paper_2506_04763_gb300 import inputs as I
        self.O = O
        O.set_threads(host_cores())
        prob = I.lognormal_lenses_box(nvert)
        self.m = O.Model(prob)
        self.F, J, md = O.assemble(self.m, prob["u0"])
        self.A = O.make_A(J, md, 1.0 / prob["H"])
        del J
        self.gm = O.GMG(3, self.m.n, self.A, prob["dir"], I.levels_for(nvert),
                        smoother=O.GS8 if smoother == "gs8" else O.JACOBI)
        self.dof = 2 * self.m.nv

    def solve(self, threads):
        self.O.set_threads(threads)
        t0 = time.perf_counter()
        x, info = self.O.bicgstab(3, self.m.n, self.A, self.gm, self.F, rtol=RTOL, maxit=200)
        dt = time.perf_counter() - t0
        return self.dof / dt, dt, info["iterations"]


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.build()
    cores = host_cores()
    sample = OracleSample(a.sample_nvert, a.smoother)
    vals = []
    for k in range(a.warmup + a.steps):
        v, dt, it = sample.solve(cores)
        if k >= a.warmup:
            vals.append((v, dt, it))
    value = statistics.median([v for v, _, _ in vals])
    ms = statistics.median([dt for _, dt, _ in vals]) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lognormal-lenses box recipe (lognormal K seed 2 + 6 lenses), %d^3 vertices, FP64 "
                                   "BiCGSTAB + FP64 GMG (8-colour GS V(2,2)), rel.res 1e-10" % a.sample_nvert,
                       "dofs": 2 * a.sample_nvert ** 3},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": cores, "kind": "oracle",
                             "sample": "oracle solve of the same recipe at %d^3 vertices (set-up excluded), OpenMP "
                                       "over vertices on %d host cores" % (a.sample_nvert, cores)},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ multi-rank helpers
def per_class_frac(v, hbm):
    return round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm, 4) if v["ms"] > 0 else None


def max_over_ranks(ms, world, device=None):
    """The job's time is its slowest rank's: MAX all-reduce of a per-rank time
    (ms) over the process group; a single process returns ms unchanged."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, ms):
    """Whole-job throughput: every rank solves its own replica (weak scaling),
    so the job processes world x units in the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


# ------------------------------------------------------------------ GPU arm
def main():
    a = args_()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    import __graft_entry__ as G
    import paper_2506_04763_gb300 as rf
    from paper_2506_04763_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if rank == 0:
        G.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    fma_rate = rf.rf_fp64_fma_rate()        # FP64 FMA/s of this GPU, measured here
    fp64_peak_tflops = 2.0 * fma_rate / 1e12

    prob = I.lognormal_lenses_box(a.nvert)
    L = I.levels_for(a.nvert)
    g = rf.Grid(prob)
    dof = 2 * g.nv
    u = torch.tensor(prob["u0"], device=dev)
    F = torch.empty_like(u)
    shift = 1.0 / prob["H"]

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # assembly (K0..K1): J, M, F(u0)
    g.assemble(u, True, F)
    e0, e1 = ev(), ev()
    e0.record(stream)
    g.assemble(u, True, F)
    e1.record(stream)
    torch.cuda.synchronize()
    asm_ms = e0.elapsed_time(e1)

    def setup(precision):
        torch.cuda.synchronize()
        s0, s1 = ev(), ev()
        s0.record(stream)
        g.gmg_setup([shift], rf.gmg_opts(L, a.smoother, precision=precision, autotune=a.autotune))
        s1.record(stream)
        torch.cuda.synchronize()
        return s0.elapsed_time(s1)

    x = torch.empty_like(F)

    def timed(nsteps, profile=False, outer=None):
        outer = outer or a.outer
        infos = []
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            # the profiled iteration graph (with event nodes) is captured on its
            # first use: do that outside the timed region
            g.profile(1)
            g.solve(0, F, x, rtol=RTOL, max_it=500, outer=outer)
            torch.cuda.synchronize()
            g.profile(1)
        l0 = rf.rf_launch_count()
        t0, t1 = ev(), ev()
        t0.record(stream)
        for _ in range(nsteps):
            infos.append(g.solve(0, F, x, rtol=RTOL, max_it=500, outer=outer))
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches = rf.rf_launch_count() - l0
        prof = None
        if profile:
            g.profile(0)
            prof = g.profile_read()
        ms = max_over_ranks(t0.elapsed_time(t1) / nsteps, world, dev)
        return ms, infos, launches, prof

    # ---- headline: FP32 (or chosen) GMG
    setup_ms = setup(a.precision)
    for _ in range(a.warmup):
        g.solve(0, F, x, rtol=RTOL, max_it=500, outer=a.outer)
    clk = Clocks(local) if rank == 0 else None
    ms, infos, launches, prof = timed(a.steps, profile=True)
    clocks = clk.stop() if clk else None
    bad = [i for i in infos if i["status"] != 0 or i["relres"] > RTOL]
    if bad:
        raise SystemExit("solve did not reach rel.res %g: %s" % (RTOL, bad[0]))
    value = job_rate(world, dof, ms)
    iters = infos[-1]["iterations"]

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    b_h = torch.empty(F.numel(), dtype=torch.float64, pin_memory=True)
    b_h.copy_(F)
    x_h = torch.empty_like(b_h).pin_memory()
    bn, xn = b_h.numpy(), x_h.numpy()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    w0 = time.perf_counter()
    for _ in range(a.steps):
        g.solve(0, bn, xn, rtol=RTOL, max_it=500, outer=a.outer)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - w0) * 1e3 / a.steps, world, dev)

    # ---- roofline of the dominant kernel class, from the live event timings
    pk = peaks()
    cands = {k: v for k, v in prof.items() if k in ("spmv64", "smooth_fine", "resid_fine") and v["ms"] > 0}
    dom = max(cands, key=lambda k: cands[k]["ms"])
    dv = prof[dom]
    achieved = dv["bytes"] / (dv["ms"] / 1e3) / 1e9
    traffic = None
    form = "colour" if os.environ.get("RF_GS_PAIRS", "1") == "0" else "pair"
    if (dom == "smooth_fine" and a.smoother == "gs8" and a.precision == "fp32"
            and a.nvert in GS_TRAFFIC_PER_VERTEX[form]):
        launch_vertices = g.nv / (8.0 if form == "colour" else 4.0)
        traffic = {"bytes_per_launch": GS_TRAFFIC_PER_VERTEX[form][a.nvert] * launch_vertices,
                   "algorithmic_bytes_per_launch": GS_ALGO_PER_VERTEX * launch_vertices,
                   "launch": ("one full-sweep colour (nv/8 vertices)" if form == "colour"
                              else "one full-sweep colour pair (nv/4 vertices)"),
                   "source": "ncu capture of this size, launches in the solve's sequence"}
    # the FP64 pipe's roofline of the outer operator (FP64-pipe-bound: 108 FMA
    # per 864 B of J), against the FMA rate measured above
    sp = prof["spmv64"]
    spmv_tflops = SPMV64_FLOP_PER_VERTEX * g.nv * sp["launches"] / (sp["ms"] / 1e3) / 1e12 if sp["ms"] > 0 else None
    roofline_fp64 = {"bound": "fp64", "kernel": "spmv64", "achieved": round(spmv_tflops, 4) if spmv_tflops else None,
                     "peak": round(fp64_peak_tflops, 4), "unit": "TFLOP/s",
                     "frac": round(spmv_tflops / fp64_peak_tflops, 4) if spmv_tflops else None,
                     "flop_per_vertex": SPMV64_FLOP_PER_VERTEX,
                     "hbm_frac_same_kernel": per_class_frac(sp, pk["hbm"]),
                     "peak_source": "rf_fp64_fma_rate in this process (8 FMA chains per thread, 2 flop per FMA)"}
    k1_rate = K1_FP64_INST_PER_VERTEX * g.nv / (asm_ms / 1e3)
    roofline_fp64["k1_assembly"] = {"kernel": "k_assemble_cells", "achieved_inst_per_s": k1_rate,
                                    "peak_inst_per_s": fma_rate, "frac": round(k1_rate / fma_rate, 4),
                                    "inst_per_vertex": K1_FP64_INST_PER_VERTEX,
                                    "source": "FP64 instruction count per vertex from ncu at 129^3; time measured here"}
    shares = {k: round(v["ms"] / sum(p["ms"] for p in prof.values()), 4) for k, v in prof.items()}
    per_class = {k: {"ms_per_step": round(v["ms"] / a.steps, 3), "launches": v["launches"],
                     "GB_per_s": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None,
                     "frac_hbm": round(v["bytes"] / (v["ms"] / 1e3) / 1e9 / pk["hbm"], 3) if v["ms"] > 0 else None}
                 for k, v in prof.items()}

    # ---- variants of the same solve: all-FP64 GPU path, FP16 storage
    variants = {}
    for var in [v for v in a.variants.split(",") if v and v != "none" and v != "%s+%s" % (a.precision, a.outer)]:
        vprec, _, vout = var.partition("+")
        vout = vout or "fp64"
        if vprec == a.precision and vout == a.outer:
            continue
        name = vprec + "_gmg" + ("" if vout == "fp64" else "_" + vout + "_outer")
        try:
            vs = setup(vprec)
            g.solve(0, F, x, rtol=RTOL, max_it=500, outer=vout)
            vms, vinf, _, vprof = timed(max(1, min(3, a.steps)), profile=True, outer=vout)
        except rf.RFError as e:
            variants[name] = {"error": str(e)}
            continue
        variants[name] = {"value": world * dof / (vms / 1e3), "unit": "DoF/s", "ms_per_solve": round(vms, 2),
                                  "iterations": vinf[-1]["iterations"], "relres": vinf[-1]["relres"],
                                  "setup_ms": round(vs, 1), "time_vs_headline": round(vms / ms, 3),
                                  "per_class_ms_per_solve": {k: round(v["ms"] / len(vinf), 3)
                                                             for k, v in vprof.items()}}

    # ---- one full LIMEX step (65^3 lognormal cube, kappa = 4, FP64 throughout)
    limex = None
    try:
        if not a.limex:
            raise _Skip()
        p2 = I.lognormal_cube_65()
        g2 = rf.Grid(p2)
        u_ref = torch.tensor(p2["u0"], device=dev)
        opts2 = rf.gmg_opts(p2["nlevels"], "jacobi", precision="fp64")
        def limex_ms(env):
            saved = {k: os.environ.pop(k, None) for k in ("RF_LIMEX_BATCH", "RF_LIMEX_CONCURRENT")}
            os.environ.update(env)
            try:
                u2 = u_ref.clone()
                g2.limex_step(u2, p2["H"], kappa=4, tol=1e-3, gmg=opts2)        # warm-up
                times, inf = [], None
                for _ in range(3):
                    u2 = u_ref.clone()
                    torch.cuda.synchronize()
                    a0, a1 = ev(), ev()
                    a0.record(stream)
                    inf = g2.limex_step(u2, p2["H"], kappa=4, tol=1e-3, gmg=opts2)
                    a1.record(stream)
                    torch.cuda.synchronize()
                    times.append(a0.elapsed_time(a1))
                return statistics.median(times), inf, u2.cpu().numpy()
            finally:
                for k in ("RF_LIMEX_BATCH", "RF_LIMEX_CONCURRENT"):
                    os.environ.pop(k, None)
                os.environ.update({k: v for k, v in saved.items() if v is not None})

        lms, info2, ub = limex_ms({})
        sms, _, us = limex_ms({"RF_LIMEX_BATCH": "0", "RF_LIMEX_CONCURRENT": "0"})
        bms, _, uc = limex_ms({"RF_LIMEX_BATCH": "1"})
        dof2 = 2 * g2.nv
        limex = {"workload": "65^3 lognormal K (seed 1), one LIMEX step H = 10 s, kappa = 4 (10 stage "
                             "solves, one Jacobian), FP64 BiCGSTAB + FP64 GMG (5 levels, block Jacobi), rel.res 1e-10",
                 "ms_per_step": round(lms, 2), "dofs_per_s": dof2 / (lms / 1e3), "dofs": dof2,
                 "solves": info2["solves"], "iterations": info2["iterations"], "eps": info2["eps"],
                 "accepted": info2["accepted"], "H_new": info2["H_new"],
                 "schedule": "columns side by side on column grids and host threads (the default below 1M "
                             "vertices)",
                 "columns_sequential_ms": round(sms, 2), "batched_rounds_ms": round(bms, 2),
                 "speedup_vs_sequential": round(sms / lms, 3),
                 "bitwise_equal_to_sequential": bool(np.array_equal(ub, us) and np.array_equal(ub, uc))}
        g2.close()
    except _Skip:
        pass
    except rf.RFError as e:
        limex = {"error": str(e)}

    # ---- ensemble: 64 realisations on uneven grids, one LIMEX step each
    ensemble = None
    if a.ensemble:
        try:
            members = I.ensemble_members()
            eprobs = [I.ensemble_member(sd, nv) for sd, nv in members]
            egrids = [rf.Grid(p) for p in eprobs]
            eu0 = [torch.tensor(p["u0"], device=dev) for p in eprobs]
            egm = [rf.gmg_opts(p["nlevels"], "jacobi", precision="fp32") for p in eprobs]
            edof = sum(2 * gg.nv for gg in egrids)

            def batched():
                us = [t.clone() for t in eu0]
                torch.cuda.synchronize()
                w0 = time.perf_counter()
                st, infos = rf.limex_step_batched(egrids, us, 10.0, kappa=4, tol=1e-3, gmg=egm)
                torch.cuda.synchronize()
                return time.perf_counter() - w0, infos

            batched()                                   # warm-up (captures graphs)
            tb_s, einfo = batched()
            os.environ["RF_LIMEX_BATCH"] = "0"          # the per-problem worker threads, for comparison
            try:
                batched()
                tt_s, _ = batched()
            finally:
                os.environ.pop("RF_LIMEX_BATCH", None)
            us = [t.clone() for t in eu0]
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            for gg, uu, oo in zip(egrids, us, egm):
                gg.limex_step(uu, 10.0, kappa=4, tol=1e-3, gmg=oo)
            torch.cuda.synchronize()
            ts_s = time.perf_counter() - w0
            ensemble = {"workload": "64 lognormal realisations (seeds 100..163) on 33^3/49^3/65^3/97^3 "
                                    "(16 each), one LIMEX step each (kappa = 4, 10 solves), FP32 GMG (block "
                                    "Jacobi) / FP64 outer, rel.res 1e-10",
                        "dofs_total": edof, "stage_solves": sum(i["solves"] for i in einfo),
                        "iterations_total": sum(i["iterations"] for i in einfo),
                        "batched_s": round(tb_s, 3), "dofs_per_s_batched": edof / tb_s,
                        "sequential_s": round(ts_s, 3), "dofs_per_s_sequential": edof / ts_s,
                        "batching_speedup": round(ts_s / tb_s, 2),
                        "threads_s": round(tt_s, 3),
                        "schedule": "problems of equal grids in shared batched rounds (one launch per kernel for "
                                    "up to 64 (member, column) systems; each member's J read once per round)",
                        "accepted": sum(i["accepted"] for i in einfo)}
            for gg in egrids:
                gg.close()
        except rf.RFError as e:
            ensemble = {"error": str(e)}

    # ---- adaptive LIMEX on the DNAPL infiltration recipe, mass check
    infiltration = None
    if a.infiltration_nvert:
        try:
            g.close()
            torch.cuda.empty_cache()
            p5 = I.dnapl_infiltration(a.infiltration_nvert)
            g5 = rf.Grid(p5)
            u5 = torch.tensor(p5["u0"], device=dev)
            m0 = g5.phase_mass(u5)[1]
            q5 = float(p5["q_in"][1::2].sum())
            opts5 = rf.gmg_opts(p5["nlevels"], "gs8", precision="fp32")
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            t5, hist = g5.limex_run(u5, 10.0, steps=a.infiltration_steps, tol=1e-3, gmg=opts5, rtol=1e-10, max_it=300)
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
            m1 = g5.phase_mass(u5)[1]
            dof5 = 2 * g5.nv
            nstep = len(hist)
            infiltration = {"workload": "%d^3 DNAPL infiltration (inlet 0.1 kg m^-2 s^-1, lognormal K seed 3 + "
                                   "lenses), adaptive LIMEX kappa = 4, TOL 1e-3, H0 = 10 s, FP32 GMG (8-colour GS) / "
                                   "FP64 outer, rel.res 1e-10" % a.infiltration_nvert,
                       "accepted": sum(h["accepted"] for h in hist), "rejected": sum(1 - h["accepted"] for h in hist),
                       "t_end_s": t5, "wall_s": round(wall, 2), "ms_per_step": round(wall * 1e3 / nstep, 1),
                       "dofs_per_s_per_step": dof5 / (wall / nstep), "dofs": dof5,
                       "stage_solves": g5.last_run["solves"],
                       "iterations": g5.last_run["iterations"],
                       "napl_mass_kg": m1, "injected_kg": q5 * t5,
                       "mass_error_rel": abs(m1 - m0 - q5 * t5) / m1,
                       "H_history": [round(h["H"], 3) for h in hist],
                       "eps_history": [float("%.4g" % h["eps"]) for h in hist],
                       "note": "first %d accepted steps of the workload's 20 (bounded for the bench's time)"
                               % a.infiltration_steps}
            g5.close()
        except (rf.RFError, RuntimeError) as e:
            infiltration = {"error": str(e)}

    # ---- Case-4 analogue: fixed-step implicit Euler + Newton against adaptive
    # LIMEX over the same simulated time (the structure of the paper's Table
    # case4_2: time steps, Newton and linear iterations, wall time)
    case4 = None
    if a.case4_days > 0:
        try:
            torch.cuda.empty_cache()
            nv4 = tuple(int(t) for t in a.case4_nvert.split("x"))
            p4 = I.case4_analogue(nv4)
            T4 = a.case4_days * 86400.0
            q4 = float(p4["q_in"][1::2].sum())
            gm4 = rf.gmg_opts(p4["nlevels"], "gs8", precision="fp64")
            case4 = {"workload": "layered Case-4 analogue, %dx%d vertices (500 m x 200 m, 4 layers), NAPL injection "
                                 "0.05 PV/year, %.0f days; FP64 GMG (8-colour GS) in BiCGSTAB, linear rel.res 1e-6"
                                 % (nv4[0], nv4[1], a.case4_days)}
            g4 = rf.Grid(p4)
            u4 = torch.tensor(p4["u0"], device=dev)
            m0 = g4.phase_mass(u4)[1]
            nst = int(round(a.case4_days))
            nn = nl = 0
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            for k in range(nst):
                inf4 = g4.ie_step(u4, T4 / nst, atol=1e-8, rtol=1e-6, max_newton=50, gmg=gm4, lin_rtol=1e-6,
                                  max_it=500)
                if inf4["status"] != 0:
                    raise RuntimeError("implicit Euler step %d failed: %s" % (k, inf4))
                nn += inf4["newton"]
                nl += inf4["linear"]
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
            m1 = g4.phase_mass(u4)[1]
            s_ie = u4.cpu().numpy()[1::2]
            case4["implicit_euler"] = {"T_total_s": round(wall, 3), "time_steps": nst, "newton": nn, "linear": nl,
                                       "dt_s": T4 / nst, "mass_error_rel": abs(m1 - m0 - q4 * T4) / (q4 * T4),
                                       "tolerances": "Newton abs 1e-8 / rel 1e-6"}
            g4.close()
            g4 = rf.Grid(p4)
            u4 = torch.tensor(p4["u0"], device=dev)
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            t4, hist = g4.limex_run(u4, 32.0, t_end=T4, tol=5e-3, rho=0.75, H_max=100 * 86400.0, gmg=gm4, rtol=1e-6,
                                    max_it=500, max_rejects=1000000)
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
            m1 = g4.phase_mass(u4)[1]
            acc = sum(h["accepted"] for h in hist)
            case4["limex"] = {"T_total_s": round(wall, 3), "time_steps": acc, "rejected": len(hist) - acc,
                              "linear": g4.last_run["iterations"], "stage_solves": g4.last_run["solves"],
                              "H_max_used_s": max(h["H"] for h in hist),
                              "mass_error_rel": abs(m1 - m0 - q4 * T4) / (q4 * T4),
                              "tolerances": "TOL 5e-3, rho 0.75, H0 32 s, H_max 100 days"}
            case4["max_abs_dSn_ie_vs_limex"] = float(np.abs(s_ie - u4.cpu().numpy()[1::2]).max())
            case4["Sn_max"] = float(s_ie.max())
            g4.close()
        except (rf.RFError, RuntimeError) as e:
            case4 = {"error": str(e)}

    cpu = None
    if rank == 0 and world == 1:
        cores = host_cores()
        sample = OracleSample(a.sample_nvert, a.smoother)
        v1, dt1, it1 = sample.solve(1)
        vn, dtn, itn = sample.solve(cores)
        cpu = {"value": vn, "unit": "DoF/s", "cores": cores, "kind": "oracle",
               "sample": "oracle FP64 BiCGSTAB-GMG solve (set-up excluded) of the same recipe at %d^3 vertices "
                         "(%d DoF, %d iterations): %.2f s on %d cores (OpenMP over vertices), %.2f s on 1"
                         % (a.sample_nvert, sample.dof, itn, dtn, cores, dt1),
               "single_thread": {"value": v1, "unit": "DoF/s", "seconds": round(dt1, 3)}}
        del sample

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/%s" % a.precision.replace("fp", "f"), "data": "synthetic",
            "config": {"workload": "%d^3-vertex box, lognormal K (seed 2) + 6 lenses, A = M/h - J "
                                   "(h = 10 s) at u0, b = F(u0); FP64 BiCGSTAB (%s operator) + %s GMG (%d levels, %s, "
                                   "V(2,2)), x0 = 0, true rel.res <= 1e-10" % (a.nvert, a.outer.upper(), a.precision.upper(), L,
                                                                            "8-colour block GS" if a.smoother == "gs8" else "block Jacobi w=0.8"),
                       "dofs": dof, "vertices": [a.nvert] * 3, "levels": L, "autotune": bool(a.autotune),
                       "l2": "no flush: inputs larger than L2 (FP64 Jacobian %.1f GB)" % (dof / 2 * 864 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "iterations": iters, "relres": infos[-1]["relres"],
            "setup_ms": round(setup_ms, 1), "assembly_ms": round(asm_ms, 1),
            "stage": {"dofs_per_s": world * dof / ((asm_ms + setup_ms + ms) / 1e3), "unit": "DoF/s",
                      "ms": round(asm_ms + setup_ms + ms, 1),
                      "note": "one LIMEX stage from scratch: assembly of J, M, F + multigrid set-up + solve"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": pk["hbm"],
                         "unit": "GB/s", "frac": round(achieved / pk["hbm"], 4), "traffic": traffic,
                         "peak_source": pk["src"], "note": "of %s HBM copy bandwidth" % pk["src"]},
            "roofline_fp64": roofline_fp64,
            "fp64_peak": {"fma_per_s": fma_rate, "tflops": round(fp64_peak_tflops, 4),
                          "source": "rf_fp64_fma_rate, measured in this process"},
            "per_class": per_class, "time_shares": shares,
            "variants": variants,
            "limex_step": limex,
            "ensemble": ensemble,
            "dnapl_infiltration": infiltration,
            "case4_analogue": case4,
            "e2e": {"value": world * dof / (e2e_ms / 1e3), "unit": "DoF/s", "h2d_bytes_per_step": 16 * g.nv,
                    "d2h_bytes_per_step": 16 * g.nv},
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    g.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
