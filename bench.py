"""Benchmark: seconds per RHMC trajectory on a 32^3x8 lattice (mixed precision
vs plain FP64, both solved to 1e-10), plus the Dslash roofline.

Workload (one "step" = one trajectory through the whole hot path: heatbath
with r_{1/4}, action with r_{-1/2}, Omelyan MD with gauge and fermion forces,
FP64 link and momentum updates, Metropolis):
  32^3x8, beta = 5.5, m = 0.0075, one pseudofermion, degree-15 rationals on
  [1e-5, 64] from the library's Remez, Omelyan 2MN, tau = 1, 20 steps,
  solver tolerance 1e-10.  Start: links exp(i 0.3 H) with H Gaussian (seed
  1 + rank), then THERM pure-gauge molecular-dynamics trajectories at the same
  beta (untimed), which bring the plaquette from 0.78 to the rough, confined
  regime (~0.50) whose Dirac spectrum has the near-zero modes that set the
  solver cost of the paper's workloads, then EQUIL RHMC trajectories with the
  Metropolis test that bring the fermion part to equilibrium (untimed).
After the timed region: the same number of trajectories end to end through
the C ABI from pinned host buffers (e2e), the next trajectory (or --chain K of
them) from the same start in FP64, float-float FP64 and the timed form, one
more trajectory under CUPTI for the kernel table, the hop roofline and the
other measurements, and the FP64 oracle's cost on the host (one core and
every core).
Multi-GPU: the path does not shard (one lattice per GPU), so N ranks run N
independent replicas (different seeds) and the value is the whole-job
seconds per trajectory: max-over-ranks time / (steps * N).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 8)
BETA, MASS, TAU, NSTEPS, DEG, LO, HI, TOL = 5.5, 0.0075, 1.0, 20, 15, 1e-5, 64.0, 1e-10
ROOF_DIMS = (64, 64, 64, 16)  # working set >= 4x L2 for the Dslash roofline
THERM, THERM_STEPS = 60, 40   # pure-gauge thermalisation: trajectories, Omelyan steps (tau = 1)
# the pure-gauge stage runs at a higher beta, whose plaquette (~0.55) is near
# that of the dynamical-fermion ensemble at BETA; the RHMC trajectories at
# BETA then start close to their equilibrium
THERM_BETA = 5.7
EQUIL = 10                    # RHMC trajectories with Metropolis after it (fermion equilibration)
# DRAM bytes (read + write) per output site of k_hop<float,1> on the roofline
# lattice 64^3x16 itself, from an ncu capture of three launches
# (dram__bytes_read.sum + dram__bytes_write.sum = 884.7 MB + 43.2 MB per
# launch, 2097152 output sites); algorithmic bytes per site: 600
HOP_TRAFFIC_PER_SITE = 442.5
# total multi-shift iterations of one FP64 trajectory of this workload, as
# counted by the library's FP64 path (identical to the oracle's recursion);
# used to scale the oracle's per-iteration cost to a trajectory
REF_ITERS_PER_TRAJ = int(os.environ.get("STAG_REF_ITERS", "0")) or None
WORKLOAD = "rhmc_32x32x32x8_omelyan20_deg15_m0.0075"


def _metric():
    return "s/trajectory (RHMC 32^3x8, 1e-10 residual)"


def replica_seeds(rank):
    """Replicas (one independent chain per rank, no data-path collective):
    every seed depends on the rank."""
    return {"links": 1 + rank, "therm": 50 + rank, "rng": 100 + rank}


def max_over_ranks(t, world):
    """The slowest rank's time (all ranks receive it)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(t_max, steps, world):
    """Whole-job seconds per trajectory: N ranks each ran `steps` trajectories
    in t_max seconds."""
    return t_max / (steps * world)


def workload_config(therm=THERM, world=1, equil=EQUIL):
    """The workload as both arms report it (config)."""
    return {"workload": WORKLOAD, "lattice": list(DIMS), "beta": BETA, "mass": MASS,
            "integrator": "omelyan", "nsteps": NSTEPS, "tau": TAU, "rational_degree": DEG,
            "rational_range": [LO, HI], "tol": TOL,
            "parallelism": "replicas" if world > 1 else "single",
            "start": {"links": "exp(i 0.3 H)",
                      "thermalisation": "%d pure-gauge MD trajectories at beta %.2f (tau 1, %d Omelyan steps, "
                                        "no Metropolis)" % (therm, THERM_BETA, THERM_STEPS),
                      "equilibration": "%d RHMC trajectories with Metropolis (MD solves 1e-7, "
                                       "Metropolis solves 1e-10)" % equil},
            "l2": "working set > L2 (links fp64+fp32+bf16 ~176 MB, solver vectors ~200 MB)"}


def _params(stag, rat_hb, rat_act, mode, traj, seed):
    return stag.make_params(BETA, MASS, TAU, NSTEPS, stag.INT_OMELYAN, rat_hb, rat_act, rat_act,
                            tol_md=TOL, tol_metro=TOL, mode_md=mode, mode_metro=mode, seed=seed,
                            traj=traj)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        rows = [r.split(", ") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# algorithmic bytes per output site of one hop, by link storage: 8 links + 8
# neighbour vectors + 1 output vector
HOP_BYTES = {"f32": 8 * 48 + 9 * 24,       # 12-real FP32 links, FP32 vectors: 600
             "f32r8": 8 * 32 + 9 * 24,     # 8-real FP32 links: 472
             "bf16": 8 * 24 + 9 * 24,      # 12-real BF16 links: 408
             "f64": 8 * 96 + 9 * 48,       # 12-real FP64 links, FP64 vectors: 1200
             "f64ff": 8 * 96 + 9 * 48}     # FP32 hi + lo link words (float-float): 1200


def hop_roofline(stag, torch, dims, nrep=30, fmt="f32", L=None):
    """Average duration of the D_oe hop with the given link storage, each
    launch timed with CUDA events on the launching stream after an L2 flush
    (a write of 512 MB).  Algorithmic bytes per output site: HOP_BYTES."""
    from paper_1106_5673_gb300 import synth
    prec = {"f32": stag.PREC_F32, "f32r8": stag.PREC_F32R8, "bf16": stag.PREC_BF16, "f64": stag.PREC_F64,
            "f64ff": stag.PREC_F64FF}[fmt]
    own = L is None
    if own:
        L = stag.Lattice(dims)
        L.load_gauge(synth.near_unit_links(dims, 0.3, 5))
    dt = torch.complex128 if fmt in ("f64", "f64ff") else torch.complex64
    x = torch.from_numpy(synth.gaussian_vector(dims, 6)).cuda().to(dt)
    y = torch.empty_like(x)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        L.apply_doe(x, y, prec)
    times = []
    for _ in range(nrep):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        L.apply_doe(x, y, prec)
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b) * 1e-3)
    if own:
        L.close()
    t = statistics.mean(times)
    Vh = int(np.prod(dims)) // 2
    nb = float(HOP_BYTES[fmt])
    return {"seconds": t, "bytes": nb * Vh, "gbs": nb * Vh / t / 1e9,
            "gflops": 570.0 * Vh / t / 1e9, "dims": list(dims), "links": fmt, "bytes_per_site": nb}


# algorithmic bytes per output site of the batched refinement's kernels with
# FP32 12-real links and R right-hand sides: A = D_oe of every p_k (links once,
# 8 neighbours + 1 output per right-hand side), B3 = D_eo of every t_k with
# p_k, r_k read and w_k written, CD = r_k, p_k, x_k read and written, w_k read
def refine_bytes(kernel, R):
    return {"k_b_A": 384 + R * 216, "k_b_B3": 384 + R * 264, "k_b_CD": R * 168}[kernel]


def refine_roofline(stag, torch, dims=(64, 64, 64, 16), nrhs=4, mass=0.0075, shift=1e-4, cupti=True):
    """The batched refinement's kernels on a lattice whose working set is far
    above L2: a mixed solve of nrhs equal shifts, so that every refinement
    launch carries nrhs right-hand sides.  Per kernel: the median of its
    launches' CUPTI device times (launches issued after convergence inside a
    graph chunk return at once and fall below the median), algorithmic bytes
    per launch (refine_bytes x Vh) and their rate against the measured copy
    peak.  cupti=False runs the same solves without the profiler (for a
    capture of the same launches under ncu)."""
    from torch.profiler import ProfilerActivity, profile
    from paper_1106_5673_gb300 import synth
    torch.cuda.set_device(0)  # torch's runtime first, as in the bench's main path
    torch.zeros(1, device="cuda")
    L = stag.Lattice(dims)
    L.load_gauge(synth.near_unit_links(dims, 0.3, 5))
    x = torch.from_numpy(synth.gaussian_vector(dims, 6)).cuda()
    shifts = [shift] * nrhs
    L.multishift_solve(mass, shifts, x, tol=TOL, mode=stag.SOLVE_MIXED)  # graphs and workspaces
    torch.cuda.synchronize()
    if cupti:  # a first, throw-away profiler session (the first one in a process recorded no kernels here)
        with profile(activities=[ProfilerActivity.CUDA]):
            torch.ones(1, device="cuda").add_(1)
            torch.cuda.synchronize()
    if not cupti:
        _, info = L.multishift_solve(mass, shifts, x, tol=TOL, mode=stag.SOLVE_MIXED)
        torch.cuda.synchronize()
        L.close()
        return {"dims": list(dims), "rhs": nrhs, "refine_iters": list(info.refine_iters[:nrhs])}
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        _, info = L.multishift_solve(mass, shifts, x, tol=TOL, mode=stag.SOLVE_MIXED)
        torch.cuda.synchronize()
    durs, seen = {}, {}
    for e in prof.profiler.kineto_results.events():  # one record per kernel launch
        name = _kernel_name(e.name())
        seen[str(e.device_type())] = seen.get(str(e.device_type()), 0) + 1
        for kname in ("k_b_A", "k_b_B3", "k_b_CD"):
            if name == kname or name.startswith(kname + "<"):
                durs.setdefault(kname, []).append(e.duration_ns() * 1e-3)
    if not durs:  # fall back to the per-name averages (post-convergence launches included)
        for e in prof.key_averages():
            name = _kernel_name(e.key)
            t = getattr(e, "device_time_total", None) or e.cuda_time_total
            for kname in ("k_b_A", "k_b_B3", "k_b_CD"):
                if (name == kname or name.startswith(kname + "<")) and t > 0:
                    durs.setdefault(kname, []).extend([t / e.count] * e.count)
    Vh = int(np.prod(dims)) // 2
    peak, kind = _peaks()
    out = {"dims": list(dims), "rhs": nrhs, "refine_iters": list(info.refine_iters[:nrhs]), "records": seen,
           "max_true_resid": max(info.true_resid[:nrhs]), "peak_gbs": peak, "peak_kind": kind}
    for kname, d in durs.items():
        t = statistics.median(d) * 1e-6
        nb = refine_bytes(kname, nrhs) * Vh
        out[kname] = {"launches": len(d), "median_us": t * 1e6, "bytes": nb, "gbs": nb / t / 1e9,
                      "frac": nb / t / 1e9 / peak}
    L.close()
    return out


def link_formats(stag, torch, dims):
    """The hop with every link storage on one lattice: 12-real FP32 against
    8-real FP32 (Sec. 4.2's minimal parametrisation) and BF16, and the
    FP64-accurate forms: a separate FP64 copy (FP64 arithmetic) against the
    FP32 hi/lo word pair of Sec. 4.2 (float-float arithmetic)."""
    from paper_1106_5673_gb300 import synth
    L = stag.Lattice(dims)
    L.load_gauge(synth.near_unit_links(dims, 0.3, 5))
    out = {fmt: hop_roofline(stag, torch, dims, fmt=fmt, L=L) for fmt in ("f32", "f32r8", "bf16", "f64", "f64ff")}
    L.close()
    return out


def equilibrate(stag, L, rat_hb, rat_act, seed, ntraj):
    """RHMC trajectories with the Metropolis test (mixed mode, MD solves to
    1e-7, Metropolis solves to 1e-10) after the pure-gauge thermalisation, so
    that the fermion part of the action is in equilibrium too before anything
    is timed; returns the list of (dH, accepted)."""
    out = []
    for i in range(ntraj):
        p = stag.make_params(BETA, MASS, TAU, NSTEPS, stag.INT_OMELYAN, rat_hb, rat_act, rat_act,
                             tol_md=1e-7, tol_metro=TOL, mode_md=stag.SOLVE_MIXED,
                             mode_metro=stag.SOLVE_MIXED, seed=seed, traj=10000 + i)
        info = L.md_trajectory(p)
        out.append((info["dH"], info["accepted"]))
    return out


def compare_chain(stag, torch, L, rat_hb, rat_act, seed, traj0, ntraj, mode, forms):
    """Trajectories traj0 .. traj0+ntraj-1 of the timed chain, each run from
    the same start configuration and random numbers in every solver form
    (FP64, float-float FP64, the timed mode); the chain continues with the
    timed mode's result.  Per trajectory: dH, accept and seconds per form."""
    rows = []
    for i in range(ntraj):
        Ustart = L.store_gauge()
        row = {"traj": traj0 + i}
        for name, m in forms:
            L2 = stag.Lattice(DIMS)
            L2.load_gauge(Ustart)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = L2.md_trajectory(_params(stag, rat_hb, rat_act, m, traj0 + i, seed))
            torch.cuda.synchronize()
            row[name] = {"s": time.perf_counter() - t0, "dH": info["dH"], "accepted": info["accepted"],
                         "cg_iters": info["cg_iters"]}
            if m == mode:
                Unext = L2.store_gauge()
            L2.close()
        L.load_gauge(Unext)
        rows.append(row)
    names = [n for n, _ in forms]
    summ = {"trajectories": ntraj,
            "s_per_traj": {n: statistics.mean(r[n]["s"] for r in rows) for n in names},
            "accept_sequences": {n: [r[n]["accepted"] for r in rows] for n in names}}
    if "f64" in names:
        for n in names:
            if n != "f64":
                summ["max_abs_ddH_%s_vs_f64" % n] = max(abs(r[n]["dH"] - r["f64"]["dH"]) for r in rows)
                summ["same_accepts_%s_vs_f64" % n] = all(r[n]["accepted"] == r["f64"]["accepted"]
                                                         for r in rows)
    if "f64" in names:
        summ["f64_cg_iters"] = statistics.mean(r["f64"]["cg_iters"] for r in rows)
    summ["rows"] = rows
    return summ


def thermalise(stag, L, rat, seed, ntraj=THERM, beta=BETA):
    """Pure-gauge molecular dynamics (npf = 0, every trajectory kept) from the
    smooth start; returns the final plaquette."""
    info = None
    for i in range(ntraj):
        p = stag.make_params(beta, MASS, 1.0, THERM_STEPS, stag.INT_OMELYAN, rat, rat, rat, npf=0,
                             mode_md=stag.SOLVE_MIXED, mode_metro=stag.SOLVE_MIXED, seed=seed,
                             traj=i, no_metropolis=1)
        info = L.md_trajectory(p)
    return info["plaq"] if info else None


BATCH_LATTICES = [(16, 16, 16, 16), (24, 24, 24, 8), (32, 32, 32, 8)]
BATCH_RHS = 96  # 8 pseudofermions x 12 shifts per lattice


def batched_hop(stag, torch, nrep=10):
    """The multi-lattice batched hop: 96 right-hand sides on each of 16^4,
    24^3x8 and 32^3x8 (links exp(i 0.2 H)) in one launch, against one launch
    per lattice and one launch per right-hand side.  Algorithmic bytes: links
    384 B per output site once per lattice, 216 B per right-hand side and
    output site (8 neighbours + output, FP32)."""
    from paper_1106_5673_gb300 import synth
    lats, ins = [], []
    for i, dims in enumerate(BATCH_LATTICES):
        L = stag.Lattice(dims)
        L.load_gauge(synth.near_unit_links(dims, 0.2, 20 + i))
        g = torch.Generator(device="cuda").manual_seed(30 + i)
        x = torch.randn((BATCH_RHS, L.Vh, 3), dtype=torch.complex64, device="cuda", generator=g)
        lats.append(L)
        ins.append(x)
    outs, cfg = stag.dslash_batch(lats, ins, out_par=1)  # tunes

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(nrep):
            fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) * 1e-3 / nrep

    t_batch = timed(lambda: stag.dslash_batch(lats, ins, outs, out_par=1))
    for L, x, y in zip(lats, ins, outs):  # tune the per-lattice launches first
        stag.dslash_batch([L], [x], [y], out_par=1)
    t_per_lat = timed(lambda: [stag.dslash_batch([L], [x], [y], out_par=1)
                               for L, x, y in zip(lats, ins, outs)])
    t_per_rhs = timed(lambda: [L.apply_doe(x[j], y[j], stag.PREC_F32)
                               for L, x, y in zip(lats, ins, outs) for j in range(BATCH_RHS)])
    alg = sum(L.Vh * (384.0 + 216.0 * BATCH_RHS) for L in lats)
    for L in lats:
        L.close()
    return {"lattices": [list(d) for d in BATCH_LATTICES], "rhs_per_lattice": BATCH_RHS,
            "tuned": {"threads_per_block": cfg[0], "rhs_per_thread": cfg[1]},
            "seconds_one_launch": t_batch, "seconds_launch_per_lattice": t_per_lat,
            "seconds_launch_per_rhs": t_per_rhs, "algorithmic_bytes": alg,
            "gbs_one_launch": alg / t_batch / 1e9}


def batched_solve(stag, torch):
    """The batched workload as solves: 8 pseudofermion sources x 12 shifts
    (poles of the degree-12 x^{-1/2} approximation on [1e-4, 64]) at m 0.01
    on each of 16^4, 24^3x8 and 32^3x8 (links exp(i 0.2 H)), mixed mode to
    1e-10.  Each lattice's 8 systems advance together in one multi-system
    shifted CG (multi-RHS hops); the three lattices run one after another,
    then concurrently on three streams (host threads; the library releases
    the interpreter while it works)."""
    import threading
    from paper_1106_5673_gb300 import synth
    m = 0.01
    _, _, shifts, _ = stag.remez(-0.5, m * m, 64.0, 12)
    lats, srcs = [], []
    for i, dims in enumerate(BATCH_LATTICES):
        L = stag.Lattice(dims)
        L.load_gauge(synth.near_unit_links(dims, 0.2, 40 + i))
        lats.append(L)
        srcs.append([torch.from_numpy(synth.gaussian_vector(dims, 60 + 10 * i + j)).cuda() for j in range(8)])
    for L, b in zip(lats, srcs):  # warm-up: tuning and graph capture
        L.multishift_solve_multi(m, shifts, b, tol=1e-10, mode=stag.SOLVE_MIXED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = [L.multishift_solve_multi(m, shifts, b, tol=1e-10, mode=stag.SOLVE_MIXED) for L, b in zip(lats, srcs)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    out = [None] * len(lats)
    streams = [torch.cuda.Stream() for _ in lats]
    torch.cuda.synchronize()

    def work(i):
        with torch.cuda.stream(streams[i]):
            out[i] = lats[i].multishift_solve_multi(m, shifts, srcs[i], tol=1e-10, mode=stag.SOLVE_MIXED)
            streams[i].synchronize()

    th = [threading.Thread(target=work, args=(i,)) for i in range(len(lats))]
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    t_con = time.perf_counter() - t0
    maxres = max(inf.true_resid[k] for _, infos in out for inf in infos for k in range(len(shifts)))
    iters = [[inf.iters for inf in infos] for _, infos in res]
    for L in lats:
        L.close()
    return {"lattices": [list(d) for d in BATCH_LATTICES], "systems_per_lattice": 8, "shifts": len(shifts),
            "mass": m, "tol": 1e-10, "seconds_sequential": t_seq, "seconds_concurrent": t_con,
            "multishift_iters": iters, "max_true_resid": maxres}


def c2_solves(stag, torch, dims=(16, 16, 16, 4), nrep=3):
    """The 16^3x4 solver workload: Haar links (seeded), m = 0.05, 16
    log-spaced shifts in [1e-4, 1] added to M_ee, complex Gaussian source on
    even sites; the FP32 multi-shift with FP64-accurate refinement against
    the FP64 shifted CG (and the float-float form), every shift to 1e-10 in
    its FP64-accurate true residual.  Seconds per solve (best of nrep after a
    warm-up) and iterations."""
    from paper_1106_5673_gb300 import synth
    L = stag.Lattice(dims)
    L.load_gauge(synth.haar_links(dims, 31))
    b = torch.from_numpy(synth.gaussian_vector(dims, 32)).cuda()
    shifts = synth.log_shifts(16, 1e-4, 1.0)
    out = {"lattice": list(dims), "mass": 0.05, "shifts": 16, "tol": 1e-10}
    for name, mode in (("mixed", stag.SOLVE_MIXED), ("f64", stag.SOLVE_F64), ("ff", stag.SOLVE_F64FF)):
        L.multishift_solve(0.05, shifts, b, tol=1e-10, mode=mode)
        best = None
        for _ in range(nrep):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = L.multishift_solve(0.05, shifts, b, tol=1e-10, mode=mode)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        out[name] = {"seconds": best, "iters": info.iters, "refine_iters": sum(info.refine_iters[:16]),
                     "max_true_resid": max(info.true_resid[:16])}
    L.close()
    return out


def reversibility(stag, torch, nmd=10, ngauge=2):
    """The paper's reversibility test (Sec. 4.4) on its 4x16^3 lattice at
    beta 5.264, am 0.01335, two pseudofermions, degree-8 MD and degree-15
    Metropolis rationals, multi-step 2MN (n_md steps, ngauge gauge steps per
    position update): integrate to tau = 1, flip the momenta, integrate back;
    Delta C and Delta M per degree of freedom, FP64 and mixed mode.  Start:
    60 pure-gauge MD trajectories from exp(i 0.3 H)."""
    from paper_1106_5673_gb300 import synth
    dims, beta, m = (16, 16, 16, 4), 5.264, 0.01335
    lo, hi = m * m / 2, 64.0
    a = stag.remez(-0.25, lo, hi, 8)[:3]      # x^{-1/(2 npf)}, npf = 2
    am = stag.remez(-0.25, lo, hi, 15)[:3]
    h = stag.remez(0.125, lo, hi, 15)[:3]     # x^{+1/(4 npf)}
    L = stag.Lattice(dims)
    L.load_gauge(synth.near_unit_links(dims, 0.3, 70))
    thermalise(stag, L, a, 71, beta=beta)
    U0 = L.store_gauge()
    W0 = synth.gaussian_momenta(dims, 72)
    phis = torch.stack([L.rational_apply(m, h, L.pf_gaussian(73, 0, pf), tol=1e-10)[0] for pf in range(2)])
    dof = 4 * 8 * int(np.prod(dims))
    out = {"lattice": list(dims), "beta": beta, "mass": m, "npf": 2, "md_degree": 8, "metro_degree": 15,
           "n_md": nmd, "ngauge": ngauge, "plaquette": L.plaquette()}
    for name, mode in (("f64", stag.SOLVE_F64), ("mixed", stag.SOLVE_MIXED)):
        p = stag.make_params(beta, m, 1.0, nmd, stag.INT_OMELYAN, h, am, a, npf=2, tol_md=1e-10,
                             tol_metro=1e-10, mode_md=mode, mode_metro=mode, ngauge=ngauge)
        L.load_gauge(U0)
        L.load_momenta(W0)
        t0 = time.perf_counter()
        it, _ = L.md_integrate(p, phis)
        t_md = time.perf_counter() - t0
        L.load_momenta(-L.store_momenta())
        L.md_integrate(p, phis)
        dC = float(np.sqrt((np.abs(L.store_gauge() - U0) ** 2).sum() / dof))
        dM = float(np.sqrt(((L.store_momenta() + W0) ** 2).sum() / dof))
        out[name] = {"delta_C": dC, "delta_M": dM, "cg_iters": it, "seconds_md": t_md}
    L.close()
    return out


# the solver settings of the paper's precision study (Sec. 4.4): (name,
# Metropolis solver, r_metro, MD solver, r_md); "mixed" is the library's FP32
# form (FP32 operator and gauge force; link and momentum updates stay FP64)
PRECISION_SETTINGS = [("D1", "f64", 1e-9, "f64", 1e-9), ("D2", "f64", 1e-7, "f64", 1e-7),
                      ("D3", "f64", 1e-5, "f64", 1e-5), ("D4", "f64", 1e-3, "f64", 1e-3),
                      ("F1", "mixed", 1e-3, "mixed", 1e-3), ("MP1", "f64", 1e-9, "mixed", 1e-3),
                      ("MP2", "f64", 1e-7, "mixed", 1e-3)]


def learned_c5(stag, torch, dims=(32, 32, 32, 32), beta=5.6, mass=0.005, nrhmc=2, npairs=32, epochs=40):
    """The learned-preconditioner workload at its lattice size (32^4, beta 5.6,
    m 0.005): links from the pure-gauge thermalisation and nrhmc mixed RHMC
    trajectories with the Metropolis test (every solve to 1e-10); the network
    trained on npairs solver-generated and on npairs operator pairs for the
    lightest pole of the degree-15 x^{-1/2} rational on [1e-5, 64]; flexible
    CG with it against plain CG, both to 1e-10."""
    from paper_1106_5673_gb300 import synth
    a0, a, b, _ = stag.remez(-0.5, 1e-5, 64.0, 15)
    h = stag.remez(0.25, 1e-5, 64.0, 15)[:3]
    L = stag.Lattice(dims)
    L.load_gauge(synth.near_unit_links(dims, 0.3, 90))
    t0 = time.perf_counter()
    plaq = thermalise(stag, L, (a0, a, b), 91, beta=beta)
    dHs = []
    for i in range(nrhmc):
        p = stag.make_params(beta, mass, 1.0, NSTEPS, stag.INT_OMELYAN, h, (a0, a, b), (a0, a, b),
                             mode_md=stag.SOLVE_MIXED, mode_metro=stag.SOLVE_MIXED, seed=92, traj=i)
        dHs.append(L.md_trajectory(p)["dH"])
    t_ens = time.perf_counter() - t0
    global MASS
    saved, MASS = MASS, mass
    try:
        out = learned_preconditioner(stag, torch, L, min(b), npairs=npairs, epochs=epochs)
    finally:
        MASS = saved
    out.update({"beta": beta, "mass": mass, "ensemble": {"pure_gauge_trajectories": THERM, "rhmc_trajectories": nrhmc,
                                                         "dH": dHs, "plaquette": L.plaquette(), "seconds": t_ens,
                                                         "therm_plaquette": plaq}})
    L.close()
    return out


def precision_study(stag, torch, lattices=((16, 16, 16, 4),), scan=((12, 1), (12, 2), (12, 4), (12, 8), (6, 5),
                                                                  (24, 5)), big=(32, 32, 32, 4)):
    """The paper's precision study (Sec. 4.4): N_f = 2 (two pseudofermions,
    degree-8 MD and degree-15 Metropolis rationals), beta = 5.264,
    am = 0.01335, multi-step 2MN integrator, tau = 1.  From one thermalised
    configuration, fixed momenta and pseudofermions, every solver setting
    D1..MP2: the reversibility violations Delta C and Delta M (integrate to
    tau, flip the momenta, integrate back) and the energy violation dH of one
    trajectory from the same start and random numbers.  Then Delta M against
    the number of gauge updates n_md x dtau_f/dtau_g (MP1 setting), and the
    MP1 and D1 points on the larger lattice."""
    from paper_1106_5673_gb300 import synth
    beta, m = 5.264, 0.01335
    lo, hi = m * m / 2, 64.0
    a_md = stag.remez(-0.25, lo, hi, 8)[:3]      # x^{-1/(2 npf)}, npf = 2
    a_metro = stag.remez(-0.25, lo, hi, 15)[:3]
    h = stag.remez(0.125, lo, hi, 15)[:3]        # x^{+1/(4 npf)}
    modes = {"f64": stag.SOLVE_F64, "mixed": stag.SOLVE_MIXED}

    def params(md, r_md, metro, r_metro, nmd, ngauge, seed=81, traj=0):
        return stag.make_params(beta, m, 1.0, nmd, stag.INT_OMELYAN, h, a_metro, a_md, npf=2, tol_md=r_md,
                                tol_metro=r_metro, mode_md=modes[md], mode_metro=modes[metro], ngauge=ngauge,
                                seed=seed, traj=traj)

    def run(dims, nmd, ngauge, settings, with_dH=True):
        L = stag.Lattice(dims)
        L.load_gauge(synth.near_unit_links(dims, 0.3, 80))
        thermalise(stag, L, a_md, 83, beta=beta)
        for i in range(3):  # RHMC trajectories with Metropolis: fermions in equilibrium
            L.md_trajectory(params("mixed", 1e-7, "mixed", 1e-10, nmd, ngauge, traj=1000 + i))
        U0 = L.store_gauge()
        W0 = synth.gaussian_momenta(dims, 84)
        phis = torch.stack([L.rational_apply(m, h, L.pf_gaussian(85, 0, pf), tol=1e-10)[0] for pf in range(2)])
        dof = 4 * 8 * int(np.prod(dims))
        rows = {"lattice": list(dims), "n_md": nmd, "dtau_f_over_dtau_g": 2 * ngauge,
                "gauge_updates": nmd * 2 * ngauge, "plaquette": L.plaquette()}
        for name, metro, r_metro, md, r_md in settings:
            p = params(md, r_md, metro, r_metro, nmd, ngauge)
            L.load_gauge(U0)
            L.load_momenta(W0)
            t0 = time.perf_counter()
            it, _ = L.md_integrate(p, phis)
            t_md = time.perf_counter() - t0
            L.load_momenta(-L.store_momenta())
            L.md_integrate(p, phis)
            dC = float(np.sqrt((np.abs(L.store_gauge() - U0) ** 2).sum() / dof))
            dM = float(np.sqrt(((L.store_momenta() + W0) ** 2).sum() / dof))
            row = {"delta_C": dC, "delta_M": dM, "cg_iters_md": it, "seconds_md": t_md}
            if with_dH:
                L.load_gauge(U0)
                info = L.md_trajectory(params(md, r_md, metro, r_metro, nmd, ngauge, traj=7))
                row["dH"] = info["dH"]
            rows[name] = row
        L.close()
        return rows

    out = {"beta": beta, "mass": m, "npf": 2, "md_degree": 8, "metro_degree": 15, "integrator": "2MN multi-step",
           "settings": {n: {"metro": (me, rm), "md": (md, rd)} for n, me, rm, md, rd in PRECISION_SETTINGS}}
    out["runs"] = [run(d, 12, 5, PRECISION_SETTINGS) for d in lattices]
    mp1 = [s_ for s_ in PRECISION_SETTINGS if s_[0] == "MP1"]
    out["gauge_update_scan"] = [run(lattices[0], nmd, ng, mp1, with_dH=False) for nmd, ng in scan]
    if big:
        out["large"] = run(big, 16, 8, [s_ for s_ in PRECISION_SETTINGS if s_[0] in ("D1", "MP1")])
    return out


def learned_preconditioner(stag, torch, L, shift, npairs=16, epochs=60):
    """The gauge-covariant network preconditioner on the workload's own
    lattice and lightest pole.  Two kinds of (source, solution) pairs:
    'solved' (random b, x from the solver) and 'operator' (random x,
    b = (M_ee + shift) x, exact, no solve); the network is trained on each,
    then flexible CG with it is compared with plain CG (both FP64-accurate,
    tol 1e-10) on a fresh source."""
    from paper_1106_5673_gb300 import synth
    dims = L.dims
    b = torch.from_numpy(synth.gaussian_vector(dims, 999)).cuda()
    out = {"lattice": list(dims), "shift": shift, "pairs": npairs, "epochs": epochs}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info = stag.fcg_solve(L, None, MASS, shift, b, tol=1e-10)
    torch.cuda.synchronize()
    out["plain_cg"] = {"iters": info.iters, "seconds": time.perf_counter() - t0,
                       "true_resid": info.true_resid[0]}
    for kind in ("solved", "operator"):
        bs, xs = [], []
        t0 = time.perf_counter()
        for j in range(npairs):
            v = torch.from_numpy(synth.gaussian_vector(dims, 500 + j)).cuda()
            if kind == "solved":
                sols, _ = L.multishift_solve(MASS, [shift], v, tol=1e-8, mode=stag.SOLVE_MIXED)
                bs.append(v)
                xs.append(sols[0])
            else:
                w = L.vector()
                L.apply_M(MASS, v, w, stag.PREC_F64FF)
                bs.append(w + shift * v)
                xs.append(v)
        torch.cuda.synchronize()
        t_pairs = time.perf_counter() - t0
        net = stag.Net(L, seed=5)
        loss0 = net.loss_grad(bs, xs)
        t0 = time.perf_counter()
        loss = net.train(bs, xs, epochs=epochs, batch=4, lr=5e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = stag.fcg_solve(L, net, MASS, shift, b, tol=1e-10)
        torch.cuda.synchronize()
        out[kind] = {"seconds_pairs": t_pairs, "seconds_train": t_train, "loss_before": loss0,
                     "loss_after": loss, "fcg_iters": info.iters,
                     "fcg_seconds": time.perf_counter() - t0, "true_resid": info.true_resid[0]}
        net.close()
    return out


def _extra(fn, *a):
    """An optional measurement: its failure is recorded in the line, not fatal."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        return {"error": "%s: %s" % (type(e).__name__, e)}


def kernel_table(stag, torch, L, params, path, top=14):
    """Per-kernel device time of one trajectory from CUPTI (torch.profiler):
    launches, total, share and average per kernel name; written to `path` and
    summarised (top kernels) in the JSON line."""
    from torch.profiler import ProfilerActivity, profile
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        info = L.md_trajectory(params)
        torch.cuda.synchronize()
    rows = []
    for e in prof.key_averages():
        t = getattr(e, "device_time_total", None)
        if t is None:
            t = e.cuda_time_total
        if t > 0:
            rows.append((e.key, e.count, t))
    tot = sum(r[2] for r in rows)
    rows.sort(key=lambda r: -r[2])
    with open(path, "w") as f:
        f.write("# one trajectory (cg_iters %d, t_total %.3f s): kernel, launches, total_ms, share, avg_us\n"
                % (info["cg_iters"], info["t_total"]))
        for k, c, t in rows:
            f.write("%s\t%d\t%.3f\t%.4f\t%.3f\n" % (k, c, t / 1e3, t / tot, t / c))
    return {"source": "CUPTI via torch.profiler, one untimed trajectory after the timed region",
            "total_ms": tot / 1e3, "launches": sum(r[1] for r in rows),
            "top": [{"kernel": _kernel_name(k), "launches": c, "ms": t / 1e3, "share": t / tot,
                     "avg_us": t / c} for k, c, t in rows[:top]]}


def _kernel_name(k):
    """Kernel name without namespace prefix and argument list."""
    k = k.replace("(anonymous namespace)::", "")
    if k.startswith("void "):
        k = k[5:]
    depth, out = 0, []
    for ch in k:
        depth += (ch == "<") - (ch == ">")
        if ch == "(" and depth == 0:
            break
        out.append(ch)
    return "".join(out)


def cpu_samples_all_cores(iters_per_traj, n_force, nrep=1):
    """nrep cpu_sample runs with the oracle's all-cores build (OpenMP over
    its site loops, identical arithmetic), in a child process with one thread
    per host core; the start links are the smooth start of the workload (the
    sample's cost does not depend on them).  Returns the list of samples."""
    ncores = os.cpu_count() or 1
    code = ("import json, sys; sys.path.insert(0, %r); import bench, oracle as O; "
            "from paper_1106_5673_gb300 import synth; O.build(openmp=True); "
            "g = json.load(open(%r))['p-1/2_d15_1e-5']; "
            "U = synth.near_unit_links(bench.DIMS, 0.3, 1); "
            "print(json.dumps([bench.cpu_sample(U, (g['a0'], g['a'], g['b']), %d, %d) for _ in range(%d)]))"
            % (ROOT, os.path.join(ROOT, "tests", "golden", "rationals.json"), iters_per_traj, n_force, nrep))
    env = dict(os.environ, ORACLE_OPENMP="1", OMP_NUM_THREADS=str(ncores))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle all-cores sample failed: %s" % r.stderr.strip()[-300:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    for o in out:
        o["cores"] = ncores
        o["sample"] = o["sample"].replace("on 1 host core", "on %d host cores (OpenMP build)" % ncores)
    return out


def cpu_sample(U, rat_act, iters_per_traj, n_force):
    """The FP64 oracle on the host: a bounded sample of the trajectory's work,
    scaled to seconds per trajectory."""
    import oracle as O
    from paper_1106_5673_gb300 import synth
    O.build()
    dims = DIMS
    a0, a, b = rat_act
    phi = synth.gaussian_vector(dims, 7)
    t0 = time.perf_counter()
    nit = 6
    _, _, tot, _ = O.multishift(dims, U, MASS, np.array(b), phi, tol=1e-30, maxit=nit)
    t_iter = (time.perf_counter() - t0) / max(tot, 1)
    t0 = time.perf_counter()
    O.gauge_force(dims, U, BETA)
    t_gf = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.fermion_force(dims, U, MASS, a0, a, b, phi, tol=1e-30, maxit=1)
    t_ff = time.perf_counter() - t0 - t_iter  # one solver iteration inside
    w = synth.gaussian_momenta(dims, 8)
    t0 = time.perf_counter()
    O.update_links(dims, U, w, 0.01)
    t_up = time.perf_counter() - t0
    est = iters_per_traj * t_iter + n_force * (t_gf + t_ff) + 2 * NSTEPS * t_up
    return {"value": est, "unit": "s/trajectory", "cores": 1, "kind": "oracle",
            "sample": ("oracle FP64 on 32^3x8: %d multi-shift iterations (15 shifts), 1 gauge "
                       "force, 1 fermion-force assembly, 1 link update, timed on 1 host core and "
                       "scaled by %d iterations and %d force evaluations per trajectory"
                       % (nit, iters_per_traj, n_force)),
            "parts_s": {"iter": t_iter, "gauge_force": t_gf, "fermion_force": t_ff,
                        "link_update": t_up}}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    iters = REF_ITERS_PER_TRAJ or args.ref_iters
    # every host core: the oracle's OpenMP build in a child process, with the
    # oracle's own Remez output (tests/golden/rationals.json, written by
    # tests/golden/make_rationals.py)
    vals = cpu_samples_all_cores(iters, 2 * NSTEPS + 1, args.warmup + args.steps)[args.warmup:]
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": _metric(), "value": v, "unit": "s/trajectory",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": v, "unit": "s/trajectory", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "s/trajectory", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    global NSTEPS, ROOF_DIMS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--ref-iters", type=int, default=137500,
                    help="FP64 multi-shift iterations per trajectory used to scale the oracle sample "
                         "(the library's FP64 count on the thermalised start)")
    ap.add_argument("--mode", default="mixed", choices=["mixed", "f64", "ff", "bf16"],
                    help="solver mode of the timed trajectories")
    ap.add_argument("--nsteps", type=int, default=NSTEPS,
                    help="MD steps (profiling runs only; the workload is 20)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the e2e and roofline measurements (profiling runs)")
    ap.add_argument("--roofline-only", action="store_true",
                    help="only time the FP32 hop on the roofline lattice")
    ap.add_argument("--solve-only", action="store_true",
                    help="only the workload's 15-shift mixed solve on 32^3x8 after --therm pure-gauge "
                         "trajectories (0: the smooth start), repeated --steps times (few launches: "
                         "for kernel profiles and solver timings)")
    ap.add_argument("--refine-roofline", action="store_true",
                    help="only time the batched refinement's kernels (four right-hand sides) on the "
                         "roofline lattice and print them as JSON (with --no-ktable: the same solves "
                         "without CUPTI, for ncu)")
    ap.add_argument("--roof-dims", default="64,64,64,16",
                    help="lattice of the large-lattice hop roofline, e.g. 48,48,48,16")
    ap.add_argument("--therm", type=int, default=THERM,
                    help="pure-gauge thermalisation trajectories before the warm-up")
    ap.add_argument("--profile-window", action="store_true",
                    help="bracket the first timed trajectory with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--kernel-table", default=None, metavar="FILE",
                    help="after the timed region, record one more trajectory with CUPTI "
                         "(torch.profiler) and write its per-kernel device-time table to FILE")
    ap.add_argument("--equil", type=int, default=EQUIL,
                    help="RHMC trajectories with Metropolis after the pure-gauge thermalisation "
                         "(fermion equilibration, untimed)")
    ap.add_argument("--chain", type=int, default=1,
                    help="trajectories after the timed region run from the same start in the FP64, "
                         "float-float and timed forms (dH, accept and time per form)")
    ap.add_argument("--no-ktable", action="store_true",
                    help="skip the CUPTI kernel table of one extra trajectory")
    ap.add_argument("--precision-study", action="store_true",
                    help="only run the paper's precision study (Sec. 4.4) and print it as JSON")
    ap.add_argument("--learned-c5", action="store_true",
                    help="only run the learned-preconditioner workload on 32^4 and print it as JSON")
    args = ap.parse_args()
    ROOF_DIMS = tuple(int(x) for x in args.roof_dims.split(","))
    if args.impl == "reference":
        return reference_arm(args)
    NSTEPS = args.nsteps
    if args.solve_only:
        import torch
        from paper_1106_5673_gb300 import stag, synth
        a0, a, b, _ = stag.remez(-0.5, LO, HI, DEG)
        L = stag.Lattice(DIMS)
        seeds = replica_seeds(0)
        L.load_gauge(synth.near_unit_links(DIMS, 0.3, seeds["links"]))
        if args.therm > 0:
            thermalise(stag, L, (a0, a, b), seeds["therm"], args.therm, beta=THERM_BETA)
        x = torch.from_numpy(synth.gaussian_vector(DIMS, 3)).cuda()
        rows = []
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, info = L.multishift_solve(MASS, b, x, tol=TOL, mode=stag.SOLVE_MIXED)
            torch.cuda.synchronize()
            rows.append(time.perf_counter() - t0)
        print(json.dumps({"solve_only": {"lattice": list(DIMS), "therm": args.therm, "beta_therm": THERM_BETA,
                                         "plaquette": L.plaquette(), "seconds": rows, "iters": info.iters,
                                         "iters_shift": list(info.iters_shift[:len(b)]),
                                         "refine_iters": list(info.refine_iters[:len(b)]),
                                         "max_true_resid": max(info.true_resid[:len(b)])}}))
        return 0
    if args.refine_roofline:
        import torch
        from paper_1106_5673_gb300 import stag
        print(json.dumps({"refine_roofline": refine_roofline(stag, torch, ROOF_DIMS, cupti=not args.no_ktable)}))
        return 0
    if args.learned_c5:
        import torch
        from paper_1106_5673_gb300 import stag
        print(json.dumps({"learned_c5": learned_c5(stag, torch)}))
        return 0
    if args.precision_study:
        import torch
        from paper_1106_5673_gb300 import stag
        print(json.dumps({"precision_study": precision_study(stag, torch)}))
        return 0
    if args.roofline_only:
        import torch
        from paper_1106_5673_gb300 import stag
        fmts = link_formats(stag, torch, ROOF_DIMS)
        peak, kind = _peaks()
        print(json.dumps({"roofline_only": fmts["f32"], "frac": fmts["f32"]["gbs"] / peak, "peak": peak,
                          "peak_kind": kind, "link_formats": fmts}))
        return 0

    import torch
    import torch.distributed as dist
    from paper_1106_5673_gb300 import stag, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    a0, a, b, err_act = stag.remez(-0.5, LO, HI, DEG)
    h0, ha, hb, err_hb = stag.remez(0.25, LO, HI, DEG)
    rat_act, rat_hb = (a0, a, b), (h0, ha, hb)
    L = stag.Lattice(DIMS)
    seeds = replica_seeds(rank)
    L.load_gauge(synth.near_unit_links(DIMS, 0.3, seeds["links"]))
    plaq_therm = thermalise(stag, L, rat_act, seeds["therm"], args.therm, beta=THERM_BETA)
    equil = equilibrate(stag, L, rat_hb, rat_act, seeds["rng"], args.equil)
    plaq_start = L.plaquette()
    U0 = L.store_gauge()

    MODES = {"mixed": stag.SOLVE_MIXED, "f64": stag.SOLVE_F64, "ff": stag.SOLVE_F64FF,
             "bf16": stag.SOLVE_MIXED_BF16}
    mode = MODES[args.mode]

    # warm-up trajectories (untimed), then K timed ones
    for i in range(args.warmup):
        L.md_trajectory(_params(stag, rat_hb, rat_act, mode, i, seeds["rng"]))
    n0 = L.launch_count()
    clocks = ClockSampler(_gpu_uuid(torch, local))
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = []
    for k in range(args.steps):
        if args.profile_window and k == 0:
            torch.cuda.profiler.start()
        infos.append(L.md_trajectory(_params(stag, rat_hb, rat_act, mode, args.warmup + k,
                                             seeds["rng"])))
        if args.profile_window and k == 0:
            torch.cuda.profiler.stop()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    t = max_over_ranks(e0.elapsed_time(e1) * 1e-3, world)
    launches = L.launch_count() - n0
    value = whole_job_value(t, args.steps, world)
    iters_timed = sum(i["cg_iters"] for i in infos) / len(infos)
    U_after = L.store_gauge()
    traj_next = args.warmup + args.steps

    # end to end through the C ABI, the same number of trajectories as the
    # timed region: every step copies the links from pinned host memory to
    # the device, runs the trajectory (its result, dH and the accept flag,
    # comes back to the host) and copies the links back to pinned memory
    t_e2e = None
    link_bytes = 4 * int(np.prod(DIMS)) * 9 * 16
    if not args.no_extras:
        pin_in = torch.empty((4, L.V, 3, 3), dtype=torch.complex128, pin_memory=True)
        pin_out = torch.empty((4, L.V, 3, 3), dtype=torch.complex128, pin_memory=True)
        pin_in.numpy()[...] = U0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            L.load_gauge(pin_in.numpy())
            L.md_trajectory(_params(stag, rat_hb, rat_act, mode, args.warmup + k, seeds["rng"]))
            L.store_gauge(out=pin_out.numpy())
        torch.cuda.synchronize()
        t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps, world) / world
        L.load_gauge(U_after)

    # the plain FP64 GPU form and the float-float FP64 form of the next
    # trajectories, each from the same start with the same random numbers as
    # the timed mode (the chain continues with the timed mode's result)
    compare = None
    if not args.no_fp64 and args.chain > 0:
        forms = [("f64", stag.SOLVE_F64), ("ff", stag.SOLVE_F64FF)]
        if args.mode not in ("f64", "ff"):
            forms.append((args.mode, mode))
        compare = compare_chain(stag, torch, L, rat_hb, rat_act, seeds["rng"], traj_next, args.chain, mode,
                                forms)
        compare["speedup_vs_f64"] = (compare["s_per_traj"]["f64"] / value) if world == 1 else None
        if args.chain == 1:
            compare.pop("rows")

    roof, roof_large, batch, bsolve, learned, revers = None, None, None, None, None, None
    formats, formats_workload, c2, refine_roof = None, None, None, None
    if not args.no_extras:
        roof = hop_roofline(stag, torch, DIMS)
        formats = _extra(link_formats, stag, torch, ROOF_DIMS)
        formats_workload = _extra(link_formats, stag, torch, DIMS)
        roof_large = formats["f32"] if "f32" in formats else hop_roofline(stag, torch, ROOF_DIMS)
        batch = _extra(batched_hop, stag, torch)
        bsolve = _extra(batched_solve, stag, torch)
        c2 = _extra(c2_solves, stag, torch)
        refine_roof = _extra(refine_roofline, stag, torch, ROOF_DIMS)
        revers = _extra(reversibility, stag, torch)
        learned = _extra(learned_preconditioner, stag, torch, L, min(rat_act[2]))
    peak, peak_kind = _peaks()
    ktable = None
    if not args.no_ktable:
        path = args.kernel_table or os.path.join(os.environ.get("TMPDIR", "/tmp"),
                                                 "stag_kernel_table_%d.txt" % os.getpid())
        ktable = _extra(kernel_table, stag, torch, L,
                        _params(stag, rat_hb, rat_act, mode, 998, seeds["rng"]), path)

    line = {
        "metric": _metric(), "value": value, "unit": "s/trajectory", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": dict(workload_config(args.therm, world, args.equil),
                       solver="mixed: fp32 multishift + fp64 reliable-update refinement",
                       rational_err=[err_act, err_hb], start_plaquette=plaq_start,
                       therm_plaquette=plaq_therm),
        # the FP32 even/odd hop that the solver kernels (k_ms_A/B3, k_b_A/B3)
        # share, on the roofline lattice (working set > 4x L2); algorithmic
        # bytes 600 per output site, traffic from the ncu capture
        "roofline": None if roof_large is None else {
            "bound": "hbm", "achieved": roof_large["gbs"], "peak": peak, "unit": "GB/s",
            "frac": roof_large["gbs"] / peak,
            "traffic": HOP_TRAFFIC_PER_SITE * roof_large["bytes"] / 600.0,
            "kernel": "k_hop<float,1> (D_oe, FP32 12-real links)", "dims": roof_large["dims"],
            "seconds_per_launch": roof_large["seconds"], "algorithmic_bytes": roof_large["bytes"],
            "dram_gbs": HOP_TRAFFIC_PER_SITE * roof_large["bytes"] / 600.0 / roof_large["seconds"] / 1e9,
            "gflops": roof_large["gflops"], "peak_kind": peak_kind},
        # the same kernel on the workload's lattice (its links fit in L2)
        "roofline_workload": None if roof is None else {
            "bound": "hbm", "achieved": roof["gbs"], "peak": peak, "unit": "GB/s",
            "frac": roof["gbs"] / peak, "dims": roof["dims"], "seconds_per_launch": roof["seconds"],
            "gflops": roof["gflops"]},
        "e2e": None if t_e2e is None else {
            "value": t_e2e, "unit": "s/trajectory", "h2d_bytes_per_step": link_bytes,
            "d2h_bytes_per_step": link_bytes, "steps": args.steps},
        "link_formats": None if formats is None else {
            "dims": list(ROOF_DIMS),
            **{k: {"seconds": v["seconds"], "gbs": v["gbs"], "bytes_per_site": v["bytes_per_site"],
                   "frac": v["gbs"] / peak}
               for k, v in formats.items() if isinstance(v, dict) and "gbs" in v}},
        "link_formats_workload": None if formats_workload is None else {
            "dims": list(DIMS),
            **{k: {"seconds": v["seconds"], "gbs": v["gbs"], "bytes_per_site": v["bytes_per_site"]}
               for k, v in formats_workload.items() if isinstance(v, dict) and "gbs" in v}},
        "gpu_launches": launches,
        "clocks": ck,
        "equilibration": {"trajectories": args.equil, "dH": [round(d, 4) for d, _ in equil],
                          "accepted": [a_ for _, a_ in equil]},
        "trajectories": [{k: i[k] for k in ("dH", "accepted", "plaq", "cg_iters", "n_force",
                                             "t_md", "t_total")} for i in infos],
        "mode": args.mode,
        "cg_iters_per_traj": iters_timed,
        "compare_same_start": compare,
        "kernel_table": ktable,
        "batched_hop": batch,
        "batched_solve": bsolve,
        "c2_solves": c2,
        "refine_roofline": refine_roof,
        "learned_preconditioner": learned,
        "reversibility": revers,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        iters = int((compare or {}).get("f64_cg_iters") or REF_ITERS_PER_TRAJ or args.ref_iters)
        cb = cpu_sample(U0, rat_act, iters, infos[0]["n_force"])
        cb["all_cores"] = _extra(lambda: {k: v for k, v in cpu_samples_all_cores(iters, infos[0]["n_force"])[0].items()
                                          if k in ("value", "cores", "sample")})
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    L.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
