"""Benchmark: PD iterations per second of the localized-collision PD hot path.

One step = one outer iteration of Algorithm 1 with one inner iteration
(local alpha step + forces, sparse forward substitution, point-triangle
self-contact detection on the device, contact update of Sigma, local beta
step + RHS, dense refactor + solve, bookkeeping, sparse backward
substitution) on the ~598K-tet elbow with 5% collision-prone nodes, the
joint flexed 40 degrees past the rest L so the crease surfaces are in
contact.  `value` is device-timed with every input resident in HBM; `e2e`
repeats the measurement through the C ABI with host buffers (the step's
Dirichlet positions uploaded and the positions read back every step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32|tf32|bf16|pcg]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the same workload

Multi-GPU runs are independent replicas (one scene per rank, no collective on
the data path); the barrier and max-over-ranks timing follow the launcher.
"""
import argparse
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PD iters/sec at 600K tets, 5% contact DOFs; Schur refactor+solve ms at 1e-10"
UNIT = "PD iters/s"
CLOSE_ANGLE = 40.0         # the joint closed this many degrees past the rest L (flexion step 65)
PEAK_FP64_ALU = 148 * 2 * 2 * 2032e6   # SMs x DFMA/clk/SM x flops/FMA x max SM clock
# DRAM bytes of one FP64 refactor + solve at m = 6,572 (the dense group: every
# k_chol_* kernel, k_trsv_tasks, k_copy_sigma, k_contact_scatter), from the
# one-pass ncu capture summarised in profiles/fp64_step_elbow598k_launches.md
# (dram__bytes_read.sum + dram__bytes_write.sum over the group's launches).
FP64_A5_DRAM_BYTES = 9.26e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "bf16", "pcg"])
    ap.add_argument("--h", type=float, default=0.585, help="elbow voxel spacing (0.585 -> ~598K tets)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the other precision forms")
    ap.add_argument("--no-extra", action="store_true", help="skip the flexion trajectory and the lips rows")
    ap.add_argument("--train-solves", type=int, default=200, help="solves recorded to train the warm start")
    ap.add_argument("--train-steps", type=int, default=1000)
    ap.add_argument("--sweep", action="store_true",
                    help="also measure inner = 3 and 5 and the Schur refactor+solve median / p90 over repeated solves")
    ap.add_argument("--nested", action="store_true",
                    help="main timed region with pd_set_contact_nodes on the proxies (nested Schur refactorisation)")
    ap.add_argument("--config5", action="store_true",
                    help="run configuration 5 at its full size (20K method-generated solves split 18K/1K/1K, the "
                         "network trained on the device, held-out PCG iterations and ms by start) and print its "
                         "JSON instead of the bench line (about 5 minutes)")
    ap.add_argument("--profile-step", action="store_true",
                    help="after warm-up run one step between cudaProfilerStart/Stop (for ncu --profile-from-start off) "
                         "and exit; prints no measurement")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_replicas(local_ms, steps, world, dist=None, device="cpu"):
    """Replicas only: every rank ran `steps` steps of its own scene; the job's
    time is the slowest rank's (max over ranks) and the job's throughput is
    all ranks' steps over that time.  Returns (max_ms, PD iterations/s)."""
    import torch
    ms = float(local_ms)
    if dist is not None and world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1e3)


def workload_name(s, precision):
    return (f"elbow (two r=8 L=60 cylinders + joint ball, voxel h={s.info['h']}): {s.E} tets, {s.n} nodes, "
            f"m={s.m} collision-prone nodes ({100.0 * s.m / s.n:.1f}%), quasistatic, {precision} region solve, "
            f"1 outer x 1 inner iteration per step, joint closed {CLOSE_ANGLE:.0f} deg past the rest L "
            f"(flexion step {int(round(45 + CLOSE_ANGLE / 2))}), point-triangle self-contact (k=1e6) detected on "
            f"the device every inner iteration")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    """Roofline denominators measured on this part (copy bandwidth, cuBLAS
    bf16 burst), else the recorded fallback; the second value names the source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, 1800.0, "fallback"


def host_info():
    """Host cores and CPU model of this machine."""
    model = platform.processor() or ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def set_detector(sol, s):
    """Point-triangle self-contact of the two elbow segments (device detection)."""
    pa, ta, pb, tb = s.info["tri_sides"]
    sol.set_detector_triangles(pa, ta, pb, tb, s.info["tri_gap"], s.info["tri_rest_min"], s.stiffness)


def form_roofline(pd, prec, m, n_ref, refactor_ms, solve_ms, iters, k_active=0):
    """Roofline of a form's dominant work.  FP64: the dense refactorisation
    (n_ref^3 / 3 flop) against the derived FP64 ALU peak.  Low-precision forms:
    the same algorithmic flops against the tensor peak of the operand type
    (TF32 = bf16 measured x the nominal 1.1 / 2.25 ratio).  PCG: the bytes its
    iterations stream (FP32 hi/lo Sigma_0 and the FP32 inverse, 12 m^2 B per
    iteration) against the measured HBM bandwidth."""
    hbm, bf16, src = measured_peaks()
    if prec == pd.PCG_WARM:
        if solve_ms <= 0:
            return None
        # per iteration: Sigma_0 as an FP32 pair (8 m^2 B), the FP32 inverse
        # (4 m^2 B) and, with the capacitance correction, the FP32 rows Y (4 k m B)
        ach = iters * (12.0 * m * m + 4.0 * k_active * m) / (solve_ms / 1e3) / 1e9
        return {"bound": "hbm", "work": "PCG iterations (k_symv_df + k_minv_apply%s)" % (
                    " + k_cap_part, k = %d" % k_active if k_active else ""),
                "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_source": src}
    if refactor_ms <= 0:
        return None
    ach = n_ref ** 3 / 3.0 / (refactor_ms / 1e3) / 1e12
    if prec == pd.FP64:
        peak, bound, ps = PEAK_FP64_ALU / 1e12, "alu", "derived FP64 DFMA peak"
    elif prec == pd.BF16_IR:
        peak, bound, ps = bf16, "tensor", src + " bf16"
    else:
        peak, bound, ps = bf16 * 1.1 / 2.25, "tensor", src + " bf16 x nominal TF32/BF16 ratio"
    return {"bound": bound, "work": "dense refactorisation, n = %d" % n_ref, "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "peak_source": ps}


def active_springs(sol):
    _, _, _, c = sol.contacts()
    return int((c > 0).sum())


def time_form(pd, sol, stream, args, fp64_ms, torch, prec, nested, cap=False):
    """Device-timed steps of one form on the current state: ms per step, PD
    iters/s, speedup over the FP64 form, the Schur contact update + refactor
    + solve time (and the refactorisation alone), refinement iterations, the
    worst relative residual and the form's roofline."""
    s = sol._scene
    for _ in range(3):
        sol.step(1)
    schur = ref = fs = iters = res = 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        sol.step(1)
        st = sol.stats()
        schur += st["ms_contact_update"] + st["ms_factor_solve"]
        ref += st["ms_refactor"]
        fs += st["ms_factor_solve"]
        iters += st["refine_iters"]
        res = max(res, st["residual"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    k = args.steps
    if nested:
        tile = 64 if prec == pd.FP64 else 128
        mp = -(-s.m // tile) * tile
        n_ref = mp - tile * ((s.m - len(s.proxies)) // tile)
    else:
        n_ref = s.m
    return {"ms_per_step": ms, "value": 1e3 / ms, "unit": UNIT, "speedup_vs_fp64": fp64_ms / ms,
            "schur_refactor_solve_ms": schur / k, "refactor_ms": ref / k, "refine_iters": iters / k,
            "max_rel_residual": res if res > 0 else None,   # None: the direct FP64 solve measures none
            "active_springs": active_springs(sol),
            "roofline": form_roofline(pd, prec, s.m, n_ref, ref / k, (fs - ref) / k, iters / k,
                                      active_springs(sol) if cap else 0)}


def time_forms(pd, sol, stream, args, fp64_ms, torch):
    """Every precision form of the region solve on the same scene and state:
    device-timed ms per step, PD iters/s, speedup over the FP64 form, the
    Schur refactor+solve time and the refinement iterations it took to reach
    the 1e-10 relative residual."""
    out = {}
    s = sol._scene
    state = sol.get_state()
    for name, prec, cap in (("fp32_ir (split-TF32 tcgen05)", pd.FP32_IR, True),
                            ("tf32_ir (TF32 tcgen05, CG-refined)", pd.TF32_IR, True),
                            ("bf16_ir (BF16 tcgen05, CG-refined)", pd.BF16_IR, True),
                            ("pcg (contact-free preconditioner M0, cold start)", pd.PCG_WARM, False),
                            ("pcg_capacitance (M0 + Woodbury correction for the active springs, cold start)",
                             pd.PCG_WARM, True)):
        sol.set_state(*state)
        sol.set_precision(prec)
        sol.set_pcg_capacitance(cap)
        out[name] = time_form(pd, sol, stream, args, fp64_ms, torch, prec, False, cap and prec == pd.PCG_WARM)
    sol.set_pcg_capacitance(True)
    # the nested Schur refactorisation on the contact-capable nodes (FP64 and split-TF32)
    npx = len(s.proxies)
    for name, prec in (("fp64_nested (FP64; Schur block of the %d contact nodes refactored, rest factored once)" % npx,
                        pd.FP64),
                       ("fp32_ir_nested (split-TF32 + IR; Schur block of the %d contact nodes refactored)" % npx,
                        pd.FP32_IR)):
        sol.set_state(*state)
        sol.set_precision(prec)
        sol.set_contact_nodes(s.proxies)
        set_detector(sol, s)
        out[name] = time_form(pd, sol, stream, args, fp64_ms, torch, prec, True)
        sol.set_contact_nodes(None)
        set_detector(sol, s)
    out.update(time_learned(pd, sol, stream, args, fp64_ms, torch, state))
    sol.set_precision(pd.FP64)
    sol.set_warm_start(0)
    sol.set_state(*state)
    sol.set_dirichlet(sol._dpos)
    set_detector(sol, s)
    return out


def schur_stats(sol, g, n):
    """Median and p90 of the Schur contact update + refactor + solve (device
    time, CUDA events inside the library) over n region solves."""
    t = []
    res = 0.0
    for _ in range(n):
        sol.schur_solve(g)
        st = sol.stats()
        t.append(st["ms_contact_update"] + st["ms_factor_solve"])
        res = max(res, st["residual"])
    t = np.sort(np.asarray(t))
    return {"median_ms": float(np.median(t)), "p90_ms": float(t[min(len(t) - 1, int(0.9 * len(t)))]),
            "solves": n, "max_rel_residual": res if res > 0 else None}   # None: the direct FP64 solve measures none


def step_rate(sol, stream, torch, steps):
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sol.step(1)
    e0.record(stream)
    for _ in range(steps):
        sol.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"ms_per_step": ms, "value": 1e3 / ms, "unit": UNIT}


TRAJ_STEPS = 71


def trajectory(pd, sol, stream, torch, forms=None):
    """The flexion of configuration 2 (Dirichlet rotation of cap B, 2 degrees
    per time step from the straight arm, 10 PD iterations per step,
    point-triangle self-contact re-detected on the device at every inner
    iteration), continued to step 70 (140 degrees, 50 past the L) because
    the synthetic arm's crease first closes into contact about 35 degrees
    past the L; with 1 and 5 inner iterations: PD iterations per second over
    the run, the step at which springs first appear and the most springs
    active at any step."""
    s = sol._scene
    out = {}
    rest = (s.X.copy(), np.zeros_like(s.X))
    forms = forms or [("split_tf32", pd.FP32_IR)]
    for fname, prec in forms:
        sol.set_precision(prec)
        for inner in (1, 5):
            sol.set_state(*rest)
            sol.set_inner_iters(inner)
            set_detector(sol, s)
            most, first = 0, None
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for step in range(TRAJ_STEPS):
                sol.set_dirichlet(s.dirichlet_positions(step))
                sol.step(10)
                k = active_springs(sol)
                most = max(most, k)
                if k > 0 and first is None:
                    first = step
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            n = 10 * TRAJ_STEPS
            out[f"{fname}_inner{inner}"] = {"pd_iterations": n, "ms_total": ms, "value": n * 1e3 / ms, "unit": UNIT,
                                            "first_contact_step": first, "max_active_springs": most}
    sol.set_inner_iters(1)
    return out


def lips_rows(pd, stream, torch, full):
    """Configuration 4: the two-slab lips scene at 2.5 / 5 / 10% collision-prone
    nodes (m = 3,125 / 6,250 / 12,500), FP64 and split-TF32 forms, about 500
    penalty springs on the facing proxies."""
    import scenes
    rows = {}
    for m in (3125, 6250, 12500):
        s = scenes.slabs(m=m)
        t0 = time.perf_counter()
        ls = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, 0.0, 0.0, inner_iters=1,
                       stream=stream.cuda_stream, timing=True, max_refine=500)
        setup_s = time.perf_counter() - t0
        # about 500 penalty springs on the facing proxies, pressed 0.1 past the gap mid-plane
        prox = s.proxies[:: max(1, len(s.proxies) // 500)][:500]
        nodes = np.full((len(prox), 4), -1, np.int32)
        nodes[:, 0] = prox
        w = np.zeros((len(prox), 4))
        w[:, 0] = 1.0
        tgt = s.X[prox] + np.where(s.X[prox, 2:3] < 9.25, 0.1, -0.1) * np.array([0.0, 0.0, 1.0])
        ls.set_dirichlet(s.dirichlet_positions(30))
        ls.set_contacts(nodes, w, tgt, np.full(len(prox), 1e6))
        gl = np.random.Generator(np.random.PCG64(6)).normal(size=(m, 3)) * 1e3
        row = {"tets": s.E, "nodes": s.n, "m": m, "region_fraction": m / s.n, "springs": len(prox),
               "setup_s": setup_s}
        for name, prec in (("fp64", pd.FP64), ("fp32_ir", pd.FP32_IR)):
            ls.set_precision(prec)
            r = step_rate(ls, stream, torch, 2 if prec == pd.FP64 else 3)
            r["schur_refactor_solve"] = schur_stats(ls, gl, (10 if full else 3) if prec == pd.FP64 else (30 if full else 10))
            row[name] = r
        ls.close()
        rows[f"m{m}"] = row
    return rows


def dynamic_rows(pd, stream, torch):
    """Backward Euler at scale: lumped mass rho * Vol / 4 per node on the
    diagonal of A (so also on Sigma_0's), dt = 1/30 s, rho = 1000, split-TF32
    form.  The elbow from the joint closed 40 degrees past the L, opened 40
    degrees and closed again (41 time steps x 10 PD iterations,
    point-triangle self-contact detected on the device at every inner
    iteration) and the lips at m = 6,250 (its 500 penalty springs, 20 time
    steps x 10 PD iterations); PD iterations per second over each run."""
    import scenes
    dt, rho = 1.0 / 30.0, 1000.0
    out = {"dt": dt, "density": rho, "form": "split-TF32 + IR"}
    s = scenes.elbow()
    t0 = time.perf_counter()
    ds = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, rho, dt, precision=pd.FP32_IR, inner_iters=1,
                   stream=stream.cuda_stream, timing=True, max_refine=500)
    setup_s = time.perf_counter() - t0
    set_detector(ds, s)
    x0, fstep = scenes.closed_pose(s, CLOSE_ANGLE)
    cycle = list(range(fstep, fstep - 21, -1)) + list(range(fstep - 19, fstep + 1))   # open 40 deg and close again
    ds.set_dirichlet(s.dirichlet_positions(fstep))
    ds.set_state(x0, np.zeros_like(x0))
    ds.step(1)                                   # warm-up
    ds.set_state(x0, np.zeros_like(x0))
    most = iters = 0
    res = 0.0
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    springs = []
    for step in cycle:
        ds.set_dirichlet(s.dirichlet_positions(step))
        ds.step(10)
        st = ds.stats()
        iters += st["refine_iters"]
        res = max(res, st["residual"])
        k = active_springs(ds)
        springs.append(k)
        most = max(most, k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    x, v = ds.get_state()
    n = 10 * len(cycle)
    out["elbow_flexion_cycle"] = {"tets": s.E, "m": s.m, "setup_s": setup_s, "time_steps": len(cycle),
                                  "what": "from the joint closed %g deg past the L (flexion step %d), opened 40 deg "
                                          "and closed again, 10 PD iterations per time step" % (CLOSE_ANGLE, fstep),
                                  "pd_iterations": n, "ms_total": ms, "value": n * 1e3 / ms, "unit": UNIT,
                                  "active_springs_first_mid_last": [springs[0], springs[len(springs) // 2],
                                                                    springs[-1]],
                                  "max_active_springs": most, "refine_iters_per_step": iters / float(len(cycle)),
                                  "max_rel_residual": res, "max_speed_end": float(np.linalg.norm(v, axis=1).max())}
    ds.close()
    s = scenes.slabs(m=6250)
    t0 = time.perf_counter()
    ds = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, rho, dt, precision=pd.FP32_IR, inner_iters=1,
                   stream=stream.cuda_stream, timing=True, max_refine=500)
    setup_s = time.perf_counter() - t0
    prox = s.proxies[:: max(1, len(s.proxies) // 500)][:500]
    nodes = np.full((len(prox), 4), -1, np.int32)
    nodes[:, 0] = prox
    w = np.zeros((len(prox), 4))
    w[:, 0] = 1.0
    tgt = s.X[prox] + np.where(s.X[prox, 2:3] < 9.25, 0.1, -0.1) * np.array([0.0, 0.0, 1.0])
    ds.set_contacts(nodes, w, tgt, np.full(len(prox), 1e6))
    ds.set_dirichlet(s.dirichlet_positions(0))
    ds.step(1)
    ds.set_state(s.X.copy(), np.zeros_like(s.X))
    torch.cuda.synchronize()
    e0.record(stream)
    for step in range(20):
        ds.set_dirichlet(s.dirichlet_positions(step))
        ds.step(10)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    out["lips_m6250"] = {"tets": s.E, "m": s.m, "setup_s": setup_s, "springs": len(prox), "pd_iterations": 200,
                         "ms_total": ms, "value": 200e3 / ms, "unit": UNIT}
    ds.close()
    return out


def sweep(pd, sol, stream, torch, args):
    """inner = 3 and 5 on the elbow and the Schur refactor+solve median / p90
    over repeated solves."""
    out = {}
    state = sol.get_state()
    g = np.random.Generator(np.random.PCG64(5)).normal(size=(sol.m, 3)) * 1e3
    for name, prec in (("fp64", pd.FP64), ("fp32_ir", pd.FP32_IR)):
        sol.set_precision(prec)
        row = {"schur_refactor_solve": schur_stats(sol, g, 50 if prec != pd.FP64 else 20)}
        for inner in (1, 3, 5):
            sol.set_state(*state)
            sol.set_inner_iters(inner)
            row[f"inner{inner}"] = step_rate(sol, stream, torch, 3)
        sol.set_inner_iters(1)
        out[name] = row
    sol.set_precision(pd.FP64)
    sol.set_state(*state)
    return out


def time_learned(pd, sol, stream, args, fp64_ms, torch, state):
    """The learned warm start: record region solves along seeded random
    indenter paths (a rigid sphere pressed into the crease surface, detected
    on the device; split-TF32 form), train the network on the device, then
    run the PCG form along a held-out indenter path from each starting point
    (zero, the previous solution, z0 = the contact-free response, the
    network) and report PCG iterations and device ms per step by start.  A
    bounded sample of the 20K-solve training run of the warmstart module."""
    from paper_2008_01541_b300 import warmstart as ws
    s = sol._scene
    # the indenter paths start from the rest state, as in the full configuration 5
    state = (s.X.copy(), np.zeros_like(s.X))
    sol.set_dirichlet(s.dirichlet_positions(s.info["rest_step"]))
    sol.clear_detector()
    t0 = time.perf_counter()
    sol.set_precision(pd.FP32_IR)
    sol.mlp_set_loss(1)
    sol.mlp_set_params(ws.he_init(0))
    sol.mlp_record(args.train_solves + 8)
    centres, radius = ws.indenter_path(s, seed=1, steps=args.train_solves)
    sol.set_state(*state)
    ws.run_path(sol, s, centres, radius)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = sol.mlp_train(args.train_steps, batch=4096, lr=1e-3, seed=2)
    train_s = time.perf_counter() - t0
    sol.mlp_record(40)
    held, radius = ws.indenter_path(s, seed=99, steps=12)
    sol.set_state(*state)
    ws.run_path(sol, s, held, radius)
    mse_net, mse_zero = sol.mlp_eval()
    sol.mlp_record(0)
    sol.set_precision(pd.PCG_WARM)
    iters, ms = {}, {}
    for name, src in (("zero", 0), ("previous", 1), ("z0", 3), ("network", 2)):
        sol.set_state(*state)
        sol.set_warm_start(src)
        ws.run_path(sol, s, held[:2], radius)          # warm-up along the first two centres
        sol.set_state(*state)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = ws.run_path(sol, s, held, radius)
        e1.record(stream)
        torch.cuda.synchronize()
        iters[name] = float(np.mean(its))
        ms[name] = e0.elapsed_time(e1) / len(held)
    r = {"ms_per_step": ms["network"], "value": 1e3 / ms["network"], "unit": UNIT,
         "speedup_vs_fp64": fp64_ms / ms["network"],
         "what": "PCG from the network's start along a held-out indenter path (sphere springs detected on the "
                 "device), %d steps of 1 outer x 1 inner iteration" % len(held),
         "heldout_pcg_iters_by_start": iters, "heldout_ms_per_step_by_start": ms,
         "train_solves": args.train_solves, "train_steps": args.train_steps, "train_loss": loss,
         "generate_s": gen_s, "train_s": train_s,
         "heldout_err_vs_z0_start": mse_net / mse_zero if mse_zero > 0 else None}
    sol.set_warm_start(0)
    return {"pcg_learned (network warm start)": r}


def run_config5(pd, s, stream, torch):
    """Configuration 5 as specified: the learned warm start trained on 18K
    method-generated region solves from seeded random indenter paths on the
    elbow, validated on 1K and tested on 1K held-out solves (disjoint paths);
    PCG iterations and device ms per step from each start, with the
    contact-free preconditioner alone and with its capacitance correction,
    beside the split-TF32 refactorisation."""
    from paper_2008_01541_b300 import warmstart as ws
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, 0.0, 0.0, stream=stream.cuda_stream,
                    timing=True, max_refine=1000)
    sol.set_dirichlet(s.dirichlet_positions(s.info["rest_step"]))
    state = sol.get_state()

    def timer(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    t0 = time.perf_counter()
    r = ws.config5(sol, s, state, timer=timer)
    r["wall_s"] = time.perf_counter() - t0
    r["workload"] = "elbow %d tets, m = %d, indenter springs detected on the device" % (s.E, s.m)
    sol.close()
    print(json.dumps({"config5": r}), flush=True)
    return 0


def frozen_contacts(sol, s):
    """The springs the device detector found in the current state, as host
    arrays in node ids (empty slots dropped)."""
    import scenes
    nodes, w, t, c = sol.contacts()
    act = c > 0
    return scenes.Contacts(nodes[act], w[act], t[act], c[act])


def _host_baseline_worker(path):
    """Child process of cpu_baseline (its BLAS / OpenMP threads fixed by the
    environment): times the oracle iteration and the LAPACK dense solve on
    the inputs saved at `path` and prints one JSON line."""
    import oracle
    import scenes
    import scipy.linalg as sla
    d = np.load(path)
    s = scenes.elbow(h=float(d["h"]))
    con = scenes.Contacts(d["nodes"], d["w"], d["target"], d["stiffness"])
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    o.x = d["x"].copy()
    t = time.perf_counter()
    o.step(1, 1, lambda x: con, d["dpos"])
    t_oracle = time.perf_counter() - t
    # LAPACK dense Cholesky + 3-RHS solve of H = Sigma_0 + C_22 (region rows)
    m = s.m
    ridx = np.full(s.n, -1, np.int64)
    ridx[s.region] = np.arange(m)
    H = d["sigma"].copy()
    for j in range(con.k):
        for a in range(con.nodes.shape[1]):
            na = con.nodes[j, a]
            if na < 0:
                continue
            for b in range(con.nodes.shape[1]):
                nb = con.nodes[j, b]
                if nb >= 0:
                    H[ridx[na], ridx[nb]] += con.stiffness[j] * con.w[j, a] * con.w[j, b]
    g = np.random.Generator(np.random.PCG64(7)).normal(size=(m, 3))
    t = time.perf_counter()
    cl = sla.cho_factor(H, lower=True, check_finite=False)
    u = sla.cho_solve(cl, g, check_finite=False)
    t_dense = time.perf_counter() - t
    print(json.dumps({"oracle_s": t_oracle, "dense_s": t_dense,
                      "dense_rel_residual": float(np.linalg.norm(g - H @ u) / np.linalg.norm(g))}), flush=True)


def cpu_baseline(scene, x_state, dpos, con, sigma):
    """Host baselines on this machine's cores, each in a child process with
    its BLAS / OpenMP threads fixed by the environment (1 and all cores).  The
    FP64 oracle as it stands: one outer x one inner iteration of the same
    scene and state (its global step a full free-node sparse LU, scipy
    SuperLU), with the springs frozen at those the device detected there.
    And the dense half of the metric: LAPACK FP64 Cholesky + solve (scipy)
    of the same H = Sigma_0 + C_22 at the same m."""
    info = host_info()
    out = dict(info)
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    np.savez(path, h=scene.info["h"], x=x_state, dpos=dpos, nodes=con.nodes, w=con.w, target=con.target,
             stiffness=con.stiffness, sigma=sigma)
    res = {}
    try:
        for cores in (1, info["nproc"]):
            env = dict(os.environ)
            for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
                env[v] = str(cores)
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--host-baseline-worker", path],
                               env=env, capture_output=True, text=True, timeout=600)
            if r.returncode != 0:
                return {"error": r.stderr[-400:], **info}
            res[cores] = json.loads(r.stdout.strip().splitlines()[-1])
    finally:
        os.unlink(path)
    a, one = res[info["nproc"]], res[1]
    out.update({"value": 1.0 / a["oracle_s"], "unit": UNIT, "cores": info["nproc"], "kind": "oracle",
                "value_1core": 1.0 / one["oracle_s"],
                "sample": "1 outer x 1 inner iteration of the same elbow state (full free-node sparse LU, scipy "
                          "SuperLU, whose sparse solve is single-threaded; BLAS and OpenMP on the given threads), "
                          "springs frozen at the %d the device detected; seconds %.1f (all cores) / %.1f (1 core)"
                          % (con.k, a["oracle_s"], one["oracle_s"])})
    out["lapack_schur_refactor_solve"] = {"ms_1core": 1e3 * one["dense_s"], "ms_all_cores": 1e3 * a["dense_s"],
                                          "m": scene.m, "rel_residual": a["dense_rel_residual"],
                                          "what": "FP64 LAPACK Cholesky (potrf) + 3-RHS solve of H = Sigma_0 + C_22"}
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, on
    the same workload, metric and unit; each timed step is one oracle PD
    iteration, and the number of timed steps is bounded so the run ends
    within a few minutes (the line reports how many were timed)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import scenes
    import oracle
    from oracle import detect
    s = scenes.elbow(h=args.h)
    o = oracle.OracleSolver(s.X, s.tets, s.dirichlet, s.region, s.mu)
    x0, fstep = scenes.closed_pose(s, CLOSE_ANGLE)
    dpos = s.dirichlet_positions(fstep)
    pa, ta, pb, tb = s.info["tri_sides"]
    gap, rmin = s.info["tri_gap"], s.info["tri_rest_min"]

    def detect_fn(x):   # the oracle's own point-triangle detection, every inner iteration
        A = detect.point_triangle_springs(pa, tb, x, s.X, gap, rmin, s.stiffness)
        B = detect.point_triangle_springs(pb, ta, x, s.X, gap, rmin, s.stiffness)
        return scenes.Contacts(*(np.concatenate([A[i], B[i]]) for i in range(4)))

    o.x = x0.copy()

    def one():
        o.step(1, 1, detect_fn, dpos)

    budget_s = 150.0
    t = time.perf_counter()
    one()                               # one untimed warm-up iteration (bounded: W is capped at 1)
    first = time.perf_counter() - t
    n = int(max(1, min(args.steps, budget_s // max(first, 1e-3))))
    t = time.perf_counter()
    for _ in range(n):
        one()
    el = time.perf_counter() - t
    v = n / el
    info = host_info()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": n, "warmup": 1, "ms_per_step": 1e3 * el / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(s, "oracle full-system FP64")},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": info["nproc"], "kind": "oracle",
                             "cpu_model": info["cpu_model"],
                             "sample": "each step = 1 outer x 1 inner oracle iteration of the full elbow scene with "
                                       "its own point-triangle detection; %d of the %d requested steps timed and 1 "
                                       "warm-up, to stay within a few minutes" % (n, args.steps)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    if len(sys.argv) == 3 and sys.argv[1] == "--host-baseline-worker":
        _host_baseline_worker(sys.argv[2])
        return 0
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2008_01541_b300 as pd
    import scenes
    prec = {"fp64": pd.FP64, "fp32": pd.FP32_IR, "tf32": pd.TF32_IR, "bf16": pd.BF16_IR,
            "pcg": pd.PCG_WARM}[args.precision]
    s = scenes.elbow(h=args.h, seed=rank)
    stream = torch.cuda.Stream()
    if args.config5:
        return run_config5(pd, s, stream, torch)
    t_setup = time.perf_counter()
    sol = pd.Solver(s.X, s.tets, s.region, s.dirichlet, s.mu, 0.0, 0.0, 0.0, precision=prec,
                    inner_iters=1, stream=stream.cuda_stream, timing=True, max_refine=500)
    setup_s = time.perf_counter() - t_setup
    sol._scene = s
    x0, fstep = scenes.closed_pose(s, CLOSE_ANGLE)
    dpos = s.dirichlet_positions(fstep)
    sol._dpos = dpos
    sol.set_state(x0, np.zeros_like(x0))
    sol.set_dirichlet(dpos)
    if args.nested:
        sol.set_contact_nodes(s.proxies)
    set_detector(sol, s)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()          # started before warm-up: NVML start-up must not fall in the timed region
    time.sleep(1.0)

    # ---- device-resident timing: inputs already in HBM, one pd_step per step
    for _ in range(max(args.warmup, 3)):
        sol.step(1)
    if args.profile_step:
        clocks.stop()
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        sol.step(1)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(json.dumps({"profile_step": True, "precision": args.precision, "nested": args.nested,
                          "kernel_launches": sol.stats()["kernel_launches"]}), flush=True)
        sol.close()
        return 0
    state = sol.get_state()
    phase_keys = ["ms_local_alpha", "ms_forward", "ms_contact_update", "ms_local_beta", "ms_factor_solve",
                  "ms_bookkeeping", "ms_backward", "ms_refactor"]
    phases = {k: 0.0 for k in phase_keys}
    launches = 0
    springs = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sol.step(1)
        st = sol.stats()
        for k in phase_keys:
            phases[k] += st[k]
        launches += st["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms, value = aggregate_replicas(e0.elapsed_time(e1), args.steps, world, dist, "cuda")
    if dist:
        dist.barrier()
    st = sol.stats()
    springs_end = active_springs(sol)

    # ---- end to end through the C ABI with host buffers: the step's Dirichlet
    # positions go up, the positions come back (contacts are detected on the device)
    sol.set_state(*state)
    dpos_seq = [np.ascontiguousarray(s.dirichlet_positions(fstep - (i % 2))) for i in range(2)]
    xbuf = np.empty((s.n, 3))
    h2d = dpos_seq[0].nbytes
    d2h = xbuf.nbytes
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        sol.set_dirichlet(dpos_seq[i % 2])
        sol.step(1)
        xbuf[:] = sol.positions()
    torch.cuda.synchronize()
    e2e_ms, e2e = aggregate_replicas(1e3 * (time.perf_counter() - t0), args.steps, world, dist, "cuda")
    sol.set_state(*state)
    sol.set_dirichlet(dpos)

    # ---- roofline of the dominant kernel group: the dense refactor + solve (a5)
    m = s.m
    flops_a5 = m ** 3 / 3.0 + 6.0 * m * m      # Cholesky m^3/3 + two triangular solves, 3 RHS
    if args.nested:   # only the trailing contact-node block is refactored (64-row tiles)
        mp = -(-m // 64) * 64
        ntr = mp - 64 * ((m - len(s.proxies)) // 64)
        flops_a5 = ntr ** 3 / 3.0 + 6.0 * m * m
    a5_ms = phases["ms_factor_solve"] / args.steps
    roof = None
    if prec == pd.FP64 and a5_ms > 0:
        ach = flops_a5 / (a5_ms / 1e3) / 1e12
        roof = {"kernel": "a5 FP64 dense refactor+solve (k_chol_diag/trsm/colupd/update/inv + k_trsv_tasks)"
                          + (", nested: trailing contact-node block" if args.nested else ""),
                "bound": "alu", "achieved": ach, "peak": PEAK_FP64_ALU / 1e12, "unit": "TFLOP/s",
                "frac": ach / (PEAK_FP64_ALU / 1e12),
                "traffic": None if args.nested else FP64_A5_DRAM_BYTES,
                "algorithmic_flop": flops_a5,
                "peak_source": "FP64 DFMA: 148 SMs x 2 FMA/clk x 2 flop x 2032 MHz (derived; "
                               "microbenchmark reached 0.95-0.99 TFLOP/s)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(s, args.precision + (" nested-Schur" if args.nested else "")),
                   "tets": s.E, "nodes": s.n, "m": s.m,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (interior factor %.0f MB, Sigma %.0f MB)" % (
                       8e-6 * st["nnz_L"], 8e-6 * m * m),
                   "spring_slots": int(st["contacts"]), "active_springs_end": springs_end},
        "schur_refactor_solve_ms": (phases["ms_contact_update"] + phases["ms_factor_solve"]) / args.steps,
        "phases_ms": {k[3:]: v / args.steps for k, v in phases.items()},
        "roofline": roof,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "setup_s": setup_s,
    }
    if not args.no_forms and not args.nested:
        line["forms"] = time_forms(pd, sol, stream, args, ms / args.steps, torch)
    if not args.no_extra and not args.nested:
        sol.set_state(*state)
        line["trajectory"] = trajectory(pd, sol, stream, torch,
                                        [("split_tf32", pd.FP32_IR), ("pcg_capacitance", pd.PCG_WARM)])
        sol.set_precision(prec)
        line["lips_config4"] = lips_rows(pd, stream, torch, args.sweep)
        line["backward_euler"] = dynamic_rows(pd, stream, torch)
    if args.sweep:
        sol.set_state(*state)
        set_detector(sol, s)
        line["sweep"] = sweep(pd, sol, stream, torch, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sol.set_state(*state)
        sol.set_dirichlet(dpos)
        set_detector(sol, s)
        sol.detect()
        con = frozen_contacts(sol, s)
        line["cpu_baseline"] = cpu_baseline(s, state[0], dpos, con, sol.schur())
    sol.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
