"""Benchmark of the disconnected-loop hot path on GB300.

One step = one complex Z2 noise vector, fully time+spin+colour diluted
(12 Lt = 384 right-hand sides on 16^3 x 32), pushed through the whole path:
noise generation -> batched mixed-precision even-odd BiCGstab to a true FP64
relative residual of 1e-10 -> loop contraction Tr[Gamma G] per site and per
time slice for Gamma = 1, g5, g1..g4.  Gauge field: U = exp(i eps H),
eps = 0.35 (seed 1), kappa = 0.120; the paper's SESAM ensemble (16^3 x 32,
Sec. II) is replaced by this synthetic field of the same shape.

Metric: RHS solves per second (whole job).  The same JSON line carries the
plain single-RHS FP64 GPU solver on a sample of the same right-hand sides,
the roofline of the dominant kernel (reduced-precision Wilson hopping term),
the oracle timed on the host cores, and an end-to-end number through the C ABI
with host buffers (gauge field uploaded from pinned host memory every step,
per-time-slice loops read back).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs independent noise vectors on its own
GPU (replicas: no data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 32)
KAPPA = 0.120
EPS = 0.35
GAUGE_SEED = 1
NOISE_SEED = 20111108
TOL = 1e-10
METRIC = "RHS solves/s at rel. residual 1e-10 (batched mixed BF16/FP32 vs plain FP64; dslash HBM GB/s)"
WORKLOAD = ("16^3x32 eps=0.35 SU(3) field (seed 1), kappa=0.120, one t+s+c-diluted complex-Z2 noise vector "
            "(384 RHS) per step: noise -> mixed-precision BiCGstab (16-bit sloppy spinors, FP32 arithmetic, "
            "FP32 reliable updates, double-float true residual) to 1e-10 -> loops")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP32 ALU peak of the hopping term: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per output (site, RHS) of the
# hop kernel each variant runs, from ncu captures of that kernel (profiles/): the solver
# runs the PLAIN, DOTR and TS epilogues 2 : 1 : 1 over the same right-hand sides.  Scaled
# to a launch by the (site, RHS) it processes; None where no capture of the current
# kernel exists.
HOP_DRAM_BYTES_PER_SITE_RHS = {
    # k_hop_pair<BF16P, *, 4, 1>, 16^3x32, 48 RHS: PLAIN 145.6, DOTR 285.8, TS 208.7
    1: (2 * 145.6 + 285.8 + 208.7) / 4,
}
HOP_KERNEL = {0: "k_hop_pair<*, *, 1, 1> (pair layout, FFMA2)", 1: "k_hop_pair<*, *, 4, 1> (pair layout, FFMA2)",
              2: "k_hop_pair<*, *, 2, 2> (pair layout, FFMA2)", 3: "k_hop_pair<*, *, 1, 4> (pair layout, FFMA2)",
              4: "k_hop_mma (pair layout, mma.sync tf32)",
              5: "k_thop (128-RHS tiles, neighbour blocks bulk-copied to shared memory, tcgen05.mma)",
              6: "k_hop_pair_pl (pair layout, FFMA2, neighbour planes staged in shared memory by cp.async)",
              7: "k_hop_pair<*, *, 4, 1, true> (pair layout, FFMA2, reconstruct-12 links)"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return parse_clock_samples(out)


def parse_clock_samples(text):
    """Median SM clock, the maximum clock and the throttle reasons seen in the CSV
    lines of `nvidia-smi --query-gpu=Clocks.Q --format=csv,noheader,nounits`."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


# --------------------------------------------------------------------- oracle
def _oracle_worker(args):
    """Solve one diluted noise source with the CPU oracle and contract it (timed)."""
    piece, = args
    import numpy as np
    from lattice_inputs import eps_su3_field
    from oracle import loops as ol, philox as oph, solver as osv
    U = eps_su3_field(DIMS, EPS, GAUGE_SEED)
    src = oph.dilute(oph.z2_noise(DIMS, NOISE_SEED, 0, 0), oph.DIL_TSC, piece)[None]
    t0 = time.perf_counter()
    phi, info = osv.solve(U, KAPPA, src, tol=TOL)
    per_site = ol.contract(src, phi)
    dt = time.perf_counter() - t0
    return dt, float(info["true_rel_residual"][0]), ol.per_timeslice(per_site)


def _oracle_warmup():
    from lattice_inputs import haar_su3_field, gaussian_spinors
    from oracle import solver as osv
    osv.solve(haar_su3_field((4, 4, 4, 4), 0), 0.125, gaussian_spinors((4, 4, 4, 4), 1, 0), tol=1e-10)


def oracle_pieces(n_rhs):
    """The diluted pieces of noise vector 0 the oracle baseline solves."""
    return [(17 * k) % (12 * DIMS[3]) for k in range(n_rhs)]


def oracle_rate(n_workers, n_rhs, with_loops=False):
    """RHS solves/s of the oracle on n_rhs sources over n_workers spawned processes."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pieces = oracle_pieces(n_rhs)
    t0 = time.perf_counter()
    with ctx.Pool(n_workers) as pool:
        res = pool.map(_oracle_worker, [(p,) for p in pieces])
    wall = time.perf_counter() - t0
    busy = max(r[0] for r in res) if n_workers >= n_rhs else wall
    info = {"rhs": n_rhs, "max_worker_s": busy, "wall_s": wall, "max_residual": max(r[1] for r in res)}
    if with_loops:
        info["loops"] = [r[2] for r in res]
    return n_rhs / busy, info


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ reference
def run_reference(args, rank, world):
    if rank != 0:
        return
    cores = host_cores()
    workers = min(cores, args.ref_rhs)
    for _ in range(args.warmup):
        _oracle_warmup()  # imports and one tiny 4^4 solve: the oracle keeps no state between steps
    vals = []
    infos = []
    for _ in range(args.steps):
        v, info = oracle_rate(workers, args.ref_rhs)
        vals.append(v)
        infos.append(info)
    total_rhs = args.ref_rhs * args.steps
    total_s = sum(i["max_worker_s"] for i in infos)
    value = total_rhs / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": args.ref_rhs, "lattice": "16x16x16x32",
                   "inputs_vs_l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "RHS solves/s", "cores": workers, "kind": "oracle",
                         "sample": f"{args.ref_rhs} of the 384 diluted sources per step, one per process, "
                                   f"FP64 numpy even-odd BiCGstab to 1e-10 + contraction"},
        "e2e": {"value": value, "unit": "RHS solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------- the gradient row of the path
def gradient_step(L, h, src, x, params, dev, stream):
    """Adjoint-solve gradient of Re sum_t w_t L_1(t) (w_t ~ N(0,1), seed 2) for the
    last step's sources and solutions: one adjoint mixed-precision solve per source,
    then the d/dkappa and d/dU contractions.  Timed with CUDA events (one warm-up)."""
    import numpy as np
    import torch
    from lattice_inputs import gaussian_weights
    V = int(np.prod(DIMS))
    coef = np.zeros((DIMS[3], 6), dtype=np.complex128)
    coef[:, 0] = gaussian_weights(DIMS[3], 2)
    dU = torch.zeros(V * 36, dtype=torch.complex128, device=dev)
    L.lqcd_gradient(h, src, x, coef, params, 1.0, dU)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    dU.zero_()
    a.record(stream)
    dk, rc, st = L.lqcd_gradient(h, src, x, coef, params, 1.0, dU)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    n = src.shape[0]
    return {"adjoint_rhs": n, "ms": ms, "adjoint_solves_per_s": n / (ms / 1e3), "status": rc,
            "max_adjoint_true_rel_residual": max(s["true_rel_residual"] for s in st),
            "dkappa": dk, "dU_norm": float(torch.linalg.vector_norm(dU).item())}


# ----------------------------------------- the other measured configurations
def config_runs(L, h, dev, stream):
    """The truncated solver method run (400 undiluted low-precision vectors to 1e-3 plus
    20 high-precision corrections to 1e-10, on the bench field) and the uneven batch of
    four lattices in one graph, each timed once after a warm-up; then each lattice of
    the batch alone (mixed solve with its hop roofline, plain FP64 sample)."""
    import numpy as np
    import torch
    from lattice_inputs import eps_su3_field, haar_su3_field
    out = {}
    V = int(np.prod(DIMS))
    solver = L.solver_params(tol=1e-10, precision=L.LQCD_PREC_MIXED_BF16)
    ps = torch.zeros((V, 6), dtype=torch.complex128, device=dev)
    pt = torch.zeros((DIMS[3], 6), dtype=torch.complex128, device=dev)
    L.lqcd_loops_stochastic(h, L.stochastic_params(7, 20, 0, 1e-3, 1e-10, L.LQCD_DILUTE_NONE, 1000), solver, ps, pt)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc, summ = L.lqcd_loops_stochastic(h, L.stochastic_params(7, 400, 20, 1e-3, 1e-10, L.LQCD_DILUTE_NONE), solver,
                                       ps, pt)
    torch.cuda.synchronize(dev)
    t = time.perf_counter() - t0
    out["tsm"] = {"lp_vectors": 400, "hp_vectors": 20, "dilution": "none", "lp_tol": 1e-3, "hp_tol": 1e-10,
                  "s": t, "solves": 420 + 20, "solves_per_s": 440 / t, "status": rc,
                  "lp_max_iterations": summ[0]["iterations"], "hp_max_iterations": summ[1]["iterations"],
                  "hp_max_true_rel_residual": summ[1]["true_rel_residual"]}
    # uneven batch: four lattices, fields and kappas in one captured graph
    specs = [((8, 8, 8, 16), "haar", 0.157, 768), ((12, 12, 12, 24), "eps", 0.115, 384),
             ((16, 16, 16, 32), "eps", 0.120, 192), ((24, 24, 24, 48), "haar", 0.157, 48)]
    handles, bufs = [], []
    batch = L.lqcd_batch_create()
    try:
        for k, (dims, kind, kappa, n) in enumerate(specs):
            U = haar_su3_field(dims, 10 + k) if kind == "haar" else eps_su3_field(dims, 0.35, 10 + k)
            hk = L.lqcd_create(dims, 0)
            handles.append(hk)
            L.lqcd_set_gauge(hk, torch.from_numpy(U.reshape(-1)).to(dev))
            L.lqcd_set_kappa(hk, kappa)
            Vl = int(np.prod(dims))
            b = torch.empty((n, Vl, 4, 3), dtype=torch.complex128, device=dev)
            npc = L.lqcd_dilution_pieces(dims, L.LQCD_DILUTE_TSC)
            for v0 in range(0, n, npc):  # several diluted vectors when n exceeds one vector's pieces
                m = min(npc, n - v0)
                L.lqcd_noise_generate(3, 0, 100 * k + v0 // npc, dims, L.LQCD_DILUTE_TSC, 0, m, b[v0:v0 + m])
            xk = torch.empty_like(b)
            bufs.append((b, xk))
            L.lqcd_batch_add(batch, hk, b, xk)
        total = sum(sp[3] for sp in specs)
        bstream = torch.cuda.Stream(device=dev)  # the batch graph is captured on a created stream
        torch.cuda.synchronize(dev)
        L.lqcd_batch_run(batch, solver, total, bstream)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rc, st = L.lqcd_batch_run(batch, solver, total, bstream)
        torch.cuda.synchronize(dev)
        t = time.perf_counter() - t0
        per, k0 = [], 0
        for dims, kind, kappa, n in specs:
            s_ = st[k0:k0 + n]
            k0 += n
            per.append({"lattice": "x".join(map(str, dims)), "field": kind, "kappa": kappa, "rhs": n,
                        "iterations_max": max(r["iterations"] for r in s_),
                        "max_true_rel_residual": max(r["true_rel_residual"] for r in s_)})
        # each lattice alone: autotuned mixed solve (solves/s, hop GB/s and fraction of
        # measured HBM) and the plain single-RHS FP64 solver on a two-source sample
        peak, _ = _peaks()
        p64 = L.solver_params(tol=1e-10, precision=L.LQCD_PREC_FP64, rhs_block=1)
        for rec, hk, (b, xk) in zip(per, handles, bufs):
            n = b.shape[0]
            L.lqcd_autotune(hk, n, solver.precision)
            L.lqcd_solve_batch(hk, b, xk, solver)  # warm-up
            torch.cuda.synchronize(dev)
            L.lqcd_profile_begin(hk)
            t0 = time.perf_counter()
            rc_k, _ = L.lqcd_solve_batch(hk, b, xk, solver)
            torch.cuda.synchronize(dev)
            tk = time.perf_counter() - t0
            pk = L.lqcd_profile_end(hk)
            hop_gbs = pk["hop_bytes"] / (pk["hop_ms"] / 1e3) / 1e9 if pk["hop_ms"] > 0 else 0.0
            x64 = torch.empty_like(b[:2])
            L.lqcd_solve_batch(hk, b[:1].contiguous(), x64[:1], p64)  # warm-up
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rc64, _ = L.lqcd_solve_batch(hk, b[:2].contiguous(), x64, p64)
            torch.cuda.synchronize(dev)
            r64 = 2 / (time.perf_counter() - t0)
            rec.update({"alone_solves_per_s": n / tk, "alone_status": rc_k, "hop_GBps": hop_gbs,
                        "hop_frac_of_hbm": hop_gbs / peak, "hop_share": pk["hop_ms"] / 1e3 / tk,
                        "fp64_plain_solves_per_s": r64, "fp64_status": rc64, "mixed_vs_plain_fp64": n / tk / r64})
            del x64
        out["uneven_batch"] = {"rhs": total, "s": t, "solves_per_s": total / t, "status": rc, "lattices": per}
    finally:
        L.lqcd_batch_destroy(batch)
        for hk in handles:
            L.lqcd_destroy(hk)
        del bufs
    return out


# --------------------------------------------- the paper's exact-loop configuration
def _exact_loops_oracle_worker(args):
    """Oracle FP64 even-odd BiCGstab on a chunk of the 4^4 point sources (timed)."""
    sites, = args
    import numpy as np
    from lattice_inputs import haar_su3_field
    from oracle.loops import point_source
    from oracle.solver import solve
    dims = (4, 4, 4, 4)
    U = haar_su3_field(dims, 0)
    lx, ly, lz, lt = dims
    src = []
    for s in sites:
        x, y, z, t = s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)
        src += [point_source(dims, (t, z, y, x), sp, c) for sp in range(4) for c in range(3)]
    src = np.stack(src)
    t0 = time.perf_counter()
    solve(U, 0.125, src, tol=1e-10)
    return time.perf_counter() - t0, len(src)


def exact_loops_4444_run(L, dev, with_oracle):
    """All 3072 point-source FP64 solves on 4^4 (Haar seed 0, kappa = 0.125) and the
    exact loops per site and per time slice: the batched FP64 solver, the plain
    single-RHS FP64 solver, and the oracle on the host cores (all 3072 sources)."""
    import numpy as np
    import torch
    from lattice_inputs import haar_su3_field
    dims = (4, 4, 4, 4)
    V = 256
    U = haar_su3_field(dims, 0)
    out = {"sources": 3072}
    h = L.lqcd_create(dims, dev.index or 0)
    try:
        L.lqcd_set_gauge(h, torch.from_numpy(U.reshape(-1)).to(dev))
        L.lqcd_set_kappa(h, 0.125)
        src = torch.empty((3072, V, 4, 3), dtype=torch.complex128, device=dev)
        L.lqcd_point_sources(h, list(range(V)), src)
        x = torch.empty_like(src)
        for name, blk in (("fp64_batched", 3072), ("fp64_plain", 1)):
            p = L.solver_params(tol=1e-10, precision=L.LQCD_PREC_FP64, rhs_block=blk)
            L.lqcd_solve_batch(h, src[:blk], x[:blk], p)  # warm-up
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rc, st = L.lqcd_solve_batch(h, src, x, p)
            torch.cuda.synchronize(dev)
            t = time.perf_counter() - t0
            out[name] = {"solves_per_s": 3072 / t, "s": t, "status": rc,
                         "max_true_rel_residual": max(r["true_rel_residual"] for r in st)}
        ps = torch.zeros((V, 6), dtype=torch.complex128, device=dev)
        pt = torch.zeros((4, 6), dtype=torch.complex128, device=dev)
        L.lqcd_loops_batch(h, src, x, 1.0, ps, pt)
        got = ps.cpu().numpy().reshape(4, 4, 4, 4, 6)
    finally:
        L.lqcd_destroy(h)
    if with_oracle:
        from oracle.loops import exact_loops_dense
        ref = exact_loops_dense(U, 0.125)
        out["loops_max_rel_err_vs_oracle_dense"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        import multiprocessing as mp
        nw = min(host_cores(), 16)
        chunks = [list(range(V))[k::nw] for k in range(nw)]
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(nw) as pool:
            res = pool.map(_exact_loops_oracle_worker, [(c,) for c in chunks])
        wall = time.perf_counter() - t0
        busy = max(r[0] for r in res)
        out["oracle"] = {"solves_per_s": 3072 / busy, "cores": nw, "max_worker_s": busy, "wall_s": wall,
                         "sample": "all 3072 point sources, split over the processes, FP64 numpy even-odd BiCGstab "
                                   "to 1e-10"}
    return out


# ------------------------------------------------- kernels beyond the step
def _event_ms(fn, stream, reps=10, warm=3):
    import torch
    for _ in range(warm):
        fn()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def _links_cpu(h, L, dev, V):
    """The context's links as a CPU array [Lt, Lz, Ly, Lx, 4, 3, 3] (zero APE steps copy them)."""
    import torch
    lx, ly, lz, lt = DIMS
    u = torch.empty(V * 36, dtype=torch.complex128, device=dev)
    L.lqcd_smear_ape(h, 0.0, 0, u)  # zero steps: copies the context's links
    return u.cpu().numpy().reshape(lt, lz, ly, lx, 4, 3, 3)


def next_rows(L, h, per_site, dev, stream, with_oracle, per_site_rhs=384):
    """Times the momentum projection, the disconnected correlator and spatially
    diluted noise on the bench lattice (after the timed step; not part of it),
    with the oracle timed beside them on the same inputs."""
    import numpy as np
    import torch
    lx, ly, lz, lt = DIMS
    V, v3 = lx * ly * lz * lt, lx * ly * lz
    out = {}
    moms = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    mo = torch.empty((len(moms), lt, 6), dtype=torch.complex128, device=dev)
    ms = _event_ms(lambda: L.lqcd_loops_momentum(h, per_site, moms, mo), stream)
    # FP64 sincospi + 6 complex FMAs per (site, momentum); per_site is read once per momentum (L2-resident)
    out["momentum_loops"] = {"n_mom": len(moms), "ms": ms, "site_momenta_per_s": V * len(moms) / (ms / 1e3),
                             "bound": "alu (FP64)",
                             "fp64_fma_gflops": V * len(moms) * 48 / (ms / 1e3) / 1e9}  # 24 FMAs per pair
    nvec = 16
    g = torch.Generator(device="cpu").manual_seed(5)
    lp = torch.randn((nvec, lt, 6), dtype=torch.complex128, generator=g).to(dev)
    lm = torch.randn((nvec, lt, 6), dtype=torch.complex128, generator=g).to(dev)
    D = torch.empty((lt, 6, 6), dtype=torch.complex128, device=dev)
    ms_c = _event_ms(lambda: L.lqcd_disconnected_correlator(lp, lm, v3, D, True), stream)
    out["correlator"] = {"n_vec": nvec, "lt": lt, "ms": ms_c}
    nz = min(384, per_site_rhs)
    buf = torch.empty((nz, V, 4, 3), dtype=torch.complex128, device=dev)
    for name, scheme in (("tsc", L.LQCD_DILUTE_TSC), ("tsc_eo", L.LQCD_DILUTE_TSC | L.LQCD_DILUTE_EO),
                         ("tsc_cube", L.LQCD_DILUTE_TSC | L.LQCD_DILUTE_CUBE)):
        ms_n = _event_ms(lambda: L.lqcd_noise_generate(NOISE_SEED, 0, 0, DIMS, scheme, 0, nz, buf), stream, reps=3)
        out[f"noise_{name}"] = {"pieces_per_vector": L.lqcd_dilution_pieces(DIMS, scheme), "chunk": nz, "ms": ms_n,
                                "write_GBps": nz * V * 192 / (ms_n / 1e3) / 1e9}
    del buf
    # smearing of connected-correlator sources: 12 point sources, APE links, F = (1 + 4 H)^50
    src12 = torch.empty((12, V, 4, 3), dtype=torch.complex128, device=dev)
    L.lqcd_point_sources(h, [0], src12)
    sm12 = torch.empty_like(src12)
    ms_ape = _event_ms(lambda: L.lqcd_smear_ape(h, 0.5, 20), stream, reps=2, warm=1)
    ms_g = _event_ms(lambda: L.lqcd_smear_gaussian(h, src12, sm12, 4.0, 50, ape_links=True, normalise=True),
                     stream, reps=2, warm=1)
    # FP64: 6 hops x 4 spins x 9 complex multiply-adds (8 flops) per (site, RHS, step)
    out["smear_gaussian"] = {"rhs": 12, "alpha": 4.0, "steps": 50, "ms": ms_g, "bound": "alu (FP64)",
                             "fp64_gflops": 12 * V * 50 * 6 * 4 * 9 * 8 / (ms_g / 1e3) / 1e9}
    out["smear_ape"] = {"alpha": 0.5, "steps": 20, "ms": ms_ape}
    if with_oracle:
        from oracle import smear as osm
        q1 = src12[:1].cpu().numpy().reshape(1, lt, lz, ly, lx, 4, 3)
        Ucpu = _links_cpu(h, L, dev, V)
        t0 = time.perf_counter()
        osm.gaussian_smear(Ucpu, q1, 4.0, 2, True)
        out["smear_gaussian"]["oracle_ms_per_rhs_step"] = 1e3 * (time.perf_counter() - t0) / 2
        out["smear_gaussian"]["ms_per_rhs_step"] = ms_g / (12 * 50)
    if with_oracle:
        from oracle import loops as olp
        ps = per_site.cpu().numpy().reshape(lt, lz, ly, lx, 6)
        t0 = time.perf_counter()
        ref = olp.momentum_loops(ps, moms)
        out["momentum_loops"]["oracle_ms"] = 1e3 * (time.perf_counter() - t0)
        got = mo.cpu().numpy()
        out["momentum_loops"]["max_rel_diff_vs_oracle"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        a, b = lp.cpu().numpy(), lm.cpu().numpy()
        t0 = time.perf_counter()
        refd = olp.disconnected_correlator(a, b, v3, True)
        out["correlator"]["oracle_ms"] = 1e3 * (time.perf_counter() - t0)
        out["correlator"]["max_rel_diff_vs_oracle"] = float(np.max(np.abs(D.cpu().numpy() - refd)) /
                                                             np.max(np.abs(refd)))
    return out


# ------------------------------------------------------------------------ ours
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    from lattice_inputs import eps_su3_field
    from paper_1108_2473_gb300 import build_lib
    build_lib.build()
    from paper_1108_2473_gb300 import lqcd as L

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    V = int(np.prod(DIMS))
    nrhs = args.nrhs
    U = eps_su3_field(DIMS, EPS, GAUGE_SEED)
    Ud = torch.from_numpy(U.reshape(-1)).to(dev)
    Uh = torch.from_numpy(U.reshape(-1)).pin_memory()
    h = L.lqcd_create(DIMS, local_rank)
    L.lqcd_set_gauge(h, Ud)
    L.lqcd_set_kappa(h, KAPPA)
    plaq = L.lqcd_plaquette(h)
    prec = L.LQCD_PREC_MIXED_FP16 if args.prec == "fp16" else L.LQCD_PREC_MIXED_BF16
    params = L.solver_params(tol=TOL, precision=prec, delta=args.delta)
    # launch-shape choice (layout, grid size, hop register budget) measured once, outside the timed region
    blocks_per_sm, hop_variant = L.lqcd_autotune(h, nrhs, prec, with_variant=True)
    src = torch.empty((nrhs, V, 4, 3), dtype=torch.complex128, device=dev)
    x = torch.empty_like(src)
    per_site = torch.zeros((V, 6), dtype=torch.complex128, device=dev)
    per_t = torch.zeros((DIMS[3], 6), dtype=torch.complex128, device=dev)
    # a created stream: the solver captures its inner iterations into a CUDA
    # graph there (the legacy default stream cannot be captured)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    def step(r, host=False):
        if host:  # end to end: a new gauge configuration arrives from pinned host memory
            L.lqcd_set_gauge(h, Uh)
        L.lqcd_noise_generate(NOISE_SEED, L.LQCD_STREAM_LP, r, DIMS, L.LQCD_DILUTE_TSC, 0, nrhs, src)
        rc, st = L.lqcd_solve_batch(h, src, x, params)
        if rc != 0:
            raise RuntimeError(f"solve failed: {L.STATUS_NAMES.get(rc, rc)} {st[:2]}")
        if host:
            pt = torch.zeros((DIMS[3], 6), dtype=torch.complex128).pin_memory()
            L.lqcd_loops_batch(h, src, x, 1.0, per_site, pt)
            return st, pt
        L.lqcd_loops_batch(h, src, x, 1.0, per_site, per_t)
        return st, None

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    from paper_1108_2473_gb300 import replicas
    # disjoint noise vectors per rank (replicas: no data-path collective)
    idx = replicas.noise_indices(rank, world, args.warmup + 2 * args.steps + 1 + args.prof_steps)
    for w in range(args.warmup):
        step(idx[w])
    # the warm-up solves may have revised the autotuner's layout choice (a pair or
    # tile computes until its slowest member converges): label what is timed
    blocks_per_sm, hop_variant = L.lqcd_tuned_choice(h, nrhs, prec)
    # ---------------------------------------------------------- timed region
    clocks = Clocks(local_rank)
    barrier()
    clocks.start()
    launches0 = L.lqcd_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters, resid = [], []
    for k in range(args.steps):
        st, _ = step(idx[args.warmup + k])
        iters += [s["iterations"] for s in st]
        resid += [s["true_rel_residual"] for s in st]
    e1.record(stream)
    barrier()
    launches = L.lqcd_launch_count() - launches0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # the hop kernel's own CUDA-event timings come from a separate profiled pass
    # (events around every hop launch; the solver then launches directly)
    L.lqcd_profile_begin(h)
    for k in range(args.prof_steps):
        step(idx[args.warmup + k])
    prof = L.lqcd_profile_end(h)
    t_max = replicas.max_over_ranks(ms, device=dev)
    solves = nrhs * args.steps * world
    value = solves / (t_max / 1e3)

    # ---------------------------------------- end to end through the C ABI
    step(idx[args.warmup + args.steps], host=True)  # warm the host path
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        _, pt = step(idx[args.warmup + args.steps + 1 + k], host=True)
        _ = pt.numpy().sum()
    barrier()
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, device=dev)
    e2e_value = solves / e2e_s

    if rank != 0:
        L.lqcd_destroy(h)
        return
    if args.skip_extras:  # profiling runs: the timed steps only
        L.lqcd_destroy(h)
        print(json.dumps({"metric": METRIC, "value": value, "unit": "RHS solves/s", "ms_per_step": t_max / args.steps,
                          "note": "--skip-extras: timed steps only, no extra rows"}), flush=True)
        return
    # the gradient row on the last step's sources and solutions (before they are reused)
    grad = gradient_step(L, h, src, x, params, dev, stream)

    # ------------------------------- plain single-RHS FP64 on a sample
    n64 = max(1, min(args.fp64_rhs, nrhs))
    xs = torch.empty((n64, V, 4, 3), dtype=torch.complex128, device=dev)
    L.lqcd_noise_generate(NOISE_SEED, L.LQCD_STREAM_LP, idx[args.warmup], DIMS, L.LQCD_DILUTE_TSC, 0, n64, src[:n64])
    p64 = L.solver_params(tol=TOL, precision=L.LQCD_PREC_FP64, rhs_block=1)
    L.lqcd_solve_batch(h, src[:1].contiguous(), xs[:1], p64)  # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc, st64 = L.lqcd_solve_batch(h, src[:n64].contiguous(), xs, p64)
    torch.cuda.synchronize(dev)
    fp64_rate = n64 / (time.perf_counter() - t0)
    extras = next_rows(L, h, per_site, dev, stream, not args.no_cpu, nrhs)
    configs = config_runs(L, h, dev, stream)
    configs["exact_loops_4x4x4x4"] = exact_loops_4444_run(L, dev, not args.no_cpu)
    gpu_piece_loops = None
    if not args.no_cpu:  # the same pieces the oracle baseline solves, for the loop error
        pcs = oracle_pieces(args.cpu_rhs)
        srcp = torch.empty((len(pcs), V, 4, 3), dtype=torch.complex128, device=dev)
        for k, pc in enumerate(pcs):
            L.lqcd_noise_generate(NOISE_SEED, L.LQCD_STREAM_LP, 0, DIMS, L.LQCD_DILUTE_TSC, pc, 1, srcp[k:k + 1])
        xp = torch.empty_like(srcp)
        L.lqcd_solve_batch(h, srcp, xp, params)
        gpu_piece_loops = []
        for k in range(len(pcs)):
            ptk = torch.zeros((DIMS[3], 6), dtype=torch.complex128, device=dev)
            L.lqcd_loops_batch(h, srcp[k:k + 1], xp[k:k + 1], 1.0, None, ptk)
            gpu_piece_loops.append(ptk.cpu().numpy())
        del srcp, xp
    L.lqcd_destroy(h)

    # ---------------------------------------------------------- roofline
    peak, peak_kind = _peaks()
    hop_s = prof["hop_ms"] / 1e3
    # algorithmic bytes of the hopping term: per output (site, RHS) one 16-bit
    # spinor read (each input read once) and one written, 2 x 48 B, plus FP16
    # reconstruct-12 links (8 x 24 B per site) once per launch
    vh = V // 2
    alg_bytes = 96.0 * prof["hop_site_rhs"] + prof["hop_launches"] * vh * 8 * 24.0
    achieved = alg_bytes / hop_s / 1e9 if hop_s > 0 else 0.0
    achieved_epi = prof["hop_bytes"] / hop_s / 1e9 if hop_s > 0 else 0.0
    traffic = None
    # the captured counters describe the BF16 kernels only
    if hop_variant in HOP_DRAM_BYTES_PER_SITE_RHS and prof["hop_launches"] > 0 and args.prec == "bf16":
        traffic = HOP_DRAM_BYTES_PER_SITE_RHS[hop_variant] * prof["hop_site_rhs"] / prof["hop_launches"]
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "traffic": traffic, "peak_kind": peak_kind,
        "bytes_model": "96 B per output (site, RHS) + 8 x 24 B reconstruct-12 links per site per launch",
        "achieved_epilogue_inclusive": achieved_epi, "frac_epilogue_inclusive": achieved_epi / peak,
        "profiled_steps": args.prof_steps,
        "kernel": f"{HOP_KERNEL.get(hop_variant, hop_variant)}, {args.prec.upper()} sloppy Wilson hopping term, "
                  f"all epilogues",
        "alg_bytes_per_launch": alg_bytes / max(prof["hop_launches"], 1),
        "site_rhs_per_launch": prof["hop_site_rhs"] / max(prof["hop_launches"], 1),
        "avg_launch_ms": prof["hop_ms"] / max(prof["hop_launches"], 1),
        "launches": prof["hop_launches"],
        "fp32_tflops": prof["hop_flops"] / hop_s / 1e12 if hop_s > 0 else 0.0,
        "fp32_frac_of_alu_peak": (prof["hop_flops"] / hop_s / 1e12) / FP32_PEAK_TFLOPS if hop_s > 0 else 0.0,
        "hop_share_of_step": hop_s / (args.prof_steps * ms / args.steps / 1e3),
    }
    # ------------------------------------------------------ CPU baseline
    cpu = None
    if not args.no_cpu:
        cores = host_cores()
        nw = min(cores, args.cpu_rhs)
        v, info = oracle_rate(nw, args.cpu_rhs, with_loops=True)
        errs = [float(np.max(np.abs(gl - ol_)) / np.max(np.abs(ol_)))
                for gl, ol_ in zip(gpu_piece_loops, info["loops"])]
        cpu = {"value": v, "unit": "RHS solves/s", "cores": nw, "kind": "oracle",
               "loop_max_rel_err_gpu_vs_oracle": max(errs),
               "sample": f"{args.cpu_rhs} of the 384 diluted sources, one per spawned process, FP64 numpy "
                         f"even-odd BiCGstab to 1e-10 + contraction; slowest process {info['max_worker_s']:.1f} s"}

    h2d = Uh.numel() * Uh.element_size()
    d2h = DIMS[3] * 6 * 16
    line = {
        "metric": METRIC, "value": value, "unit": "RHS solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{args.prec}/fp32 (Krylov) + f64 (loops, outer x)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": nrhs * world, "lattice": "16x16x16x32",
                   "precision": args.prec, "parallelism": f"replicas x{world}",
                   "inputs_vs_l2": "working set ~30 GB per step >> 129 MB L2 (no flush needed)",
                   "plaquette": plaq, "blocks_per_sm": blocks_per_sm, "hop_variant": hop_variant},
        "mixed_vs_plain_fp64": value / world / fp64_rate,
        "fp64_plain": {"value": fp64_rate, "unit": "RHS solves/s", "sample_rhs": n64,
                       "what": "plain single-RHS FP64 even-odd BiCGstab (one RHS per solve) on the first n of the "
                               "step's diluted sources: the 16^3x32 plain-FP64 configuration",
                       "iterations": [s["iterations"] for s in st64]},
        "solver": {"iterations_min": min(iters), "iterations_max": max(iters), "max_true_rel_residual": max(resid)},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "RHS solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "gradient": grad,
        "configs": configs,
        "next_rows": extras,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["fp16", "bf16"])
    ap.add_argument("--delta", type=float, default=0.05, help="reliable-update threshold of the mixed solver")
    ap.add_argument("--nrhs", type=int, default=12 * DIMS[3], help="diluted sources per step (384 = all)")
    ap.add_argument("--fp64-rhs", type=int, default=12 * DIMS[3],
                    help="right-hand sides of the plain single-RHS FP64 sample (384 = one diluted vector)")
    ap.add_argument("--prof-steps", type=int, default=1, help="steps of the profiled pass (hop roofline)")
    ap.add_argument("--cpu-rhs", type=int, default=16)
    ap.add_argument("--ref-rhs", type=int, default=16)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="stop after the timed steps and the end-to-end leg (for launch-list profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
