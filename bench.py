"""Benchmark: MG solves/s to true relative residual 1e-10 on a 256^2 lattice.

Workload: 2D U(1) staggered operator on a 256x256 periodic lattice, links from a
seeded heatbath at beta = 6 (2000 sweeps), m = 1e-3; 3-level Kaehler-Dirac
multigrid with 4x4 (KD blocks) then 2x2 aggregates and 24 then 32 null
vectors; complex128 everywhere; one Gaussian right-hand side per step.  The
multigrid setup is done once, outside the timed region, and reported apart.

One JSON line on stdout.  --impl reference times the FP64 CPU oracle instead.
Several GPUs: independent replicas (each rank solves its own right-hand
sides; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

# The oracle timings (cpu_baseline, --impl reference) are single-core: keep
# BLAS from spawning threads before numpy loads it.
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s to rel. resid 1e-10 (256², m=1e-3)"
UNIT = "solves/s"
WORKLOAD = dict(workload="KD-staggered MG solve, 2D U(1) 256x256, beta=6 (2000 heatbath sweeps), "
                         "m=1e-3, 3 levels (4x4 KD-block then 2x2 aggregates), Nv 24/32, "
                         "complex128, 1 Gaussian RHS per solve, tol 1e-10; Table kcycle "
                         "parameters except coarsest CGNE cap 2048",
                L=256, beta=6.0, sweeps=2000, mass=1e-3, levels=3, blocks=[[4, 4], [2, 2]],
                nvec=[24, 32], tol=1e-10, coarsest_maxiter=2048)
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12  # 4 FP64 flop/clk/SM (2 DFMA) x 152 SMs x 2070 MHz


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback copy bandwidth


HBM_PEAK_GBS = _hbm_peak()


def _profiled_traffic(profile: str, source: str, key: str):
    """A DRAM-traffic figure recorded in profiles/<profile> by an ncu capture,
    or None when the kernel source has changed since that capture."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        want = hashlib.sha1(open(os.path.join(ROOT, source), "rb").read()).hexdigest()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line)
    sha = fields.get(f"source_sha1 ({source})")
    if sha is None or sha.strip() != want or key not in fields:
        return None
    return float(fields[key])


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks, on every rank (x itself on one rank)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def rhs_seed(rank: int, k: int, offset: int = 0) -> int:
    """Seed of right-hand side k of a rank: replicas solve different systems."""
    return rank * 1000 + offset + k


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--L", type=int, default=WORKLOAD["L"])
    ap.add_argument("--sweeps", type=int, default=WORKLOAD["sweeps"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the mixed-precision solve measured beside the FP64 one")
    ap.add_argument("--batched-only", type=int, default=0, metavar="K",
                    help="run only K-right-hand-side batched solves on the mixed hierarchy "
                         "(one warm-up and --batch-reps timed batches; for profiling)")
    ap.add_argument("--batch-f32", action="store_true",
                    help="with --batched-only: FP32 iterates in the batched coarsest CGNE")
    ap.add_argument("--dslash-only", action="store_true",
                    help="run only the Dslash bandwidth microbenchmark")
    ap.add_argument("--batch-reps", type=int, default=3,
                    help="timed batches per batch width")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving measurement (with the options below)")
    ap.add_argument("--serving-workers", type=int, default=3)
    ap.add_argument("--serving-batch", type=int, default=8)
    ap.add_argument("--serving-rate", type=float, default=4.0)
    ap.add_argument("--serving-fp64", action="store_true",
                    help="serve with FP64 hierarchies (the plain baseline of the served form)")
    ap.add_argument("--serving-requests", type=int, default=48,
                    help="requests of the serving measurement (0: skip it)")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def gauge_and_psi0(L, beta, sweeps, device):
    import sw_inputs as si
    th = si.heatbath_u1(L, L, beta, sweeps, seed=1, device=device)
    nv = WORKLOAD["nvec"]
    b0 = WORKLOAD["blocks"][0][0]
    psi0 = [np.stack([si.gaussian_complex(si.stream_seed(5, 0, i), L * L) for i in range(nv[0])])]
    E = L // (2 * b0)
    psi0.append(np.stack([si.gaussian_complex(si.stream_seed(5, 1, i), E * E * 2 * nv[0])
                          for i in range(nv[1])]))
    return th, psi0


def rhs(seed, L):
    import sw_inputs as si
    return si.gaussian_complex(1000 + seed, L * L)


# ---------------------------------------------------------------------------- CPU oracle
COUNTS_FILE = os.path.join(ROOT, "oracle", "solve_counts_256.json")


def oracle_counts(L):
    """Application counts and wall-time ratio of the oracle's own full solve of
    this workload (written by oracle/solve_counts.py), or None for another size."""
    try:
        with open(COUNTS_FILE) as f:
            rec = json.load(f)
    except OSError:
        return None
    return rec if rec["workload"]["L"] == L else None


def oracle_hierarchy(th, m, psi0):
    """The oracle's hierarchy of this workload built with zero setup CG steps:
    the shapes and sparsity of the real one, for timing its operators."""
    from oracle import mg as omg
    return omg.Hierarchy(th, m, 3, [tuple(b) for b in WORKLOAD["blocks"]], WORKLOAD["nvec"],
                         [list(a) for a in psi0], omg.Params(setup_maxiter=0))


def oracle_solve_seconds(H, rec, reps):
    """Seconds per oracle solve from a bounded sample: `reps` applications each of
    the oracle's S, A_hat (level 2) and A_hat (level 3) timed here, weighted by
    the counts of the oracle's own full solve and scaled by that solve's ratio of
    wall time to application time.  Returns (seconds, per-application times)."""
    from oracle.solve_counts import apply_times
    ta = apply_times(H, reps)
    c = rec["counts"]
    return rec["overhead_ratio"] * sum(c[k] * ta[k] for k in c), ta


def cpu_model() -> str:
    """CPU model name of this host (lscpu, else /proc/cpuinfo) and its core count."""
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    name = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return f"{name or 'unknown'}, nproc {os.cpu_count()}"


def oracle_validation(sizes=(32, 64)):
    """Measured full single-core oracle solves at small lattices (3 levels, the
    paper's Nv 8/12, beta 6, m = 0.01, tol 1e-10), each beside the prediction
    of the model that extrapolates the 256^2 figure (application counts x
    per-application times here x the 256^2 solve's wall/application ratio)."""
    import sw_inputs as si
    from oracle import mg as omg
    from oracle.solve_counts import _Counted, apply_times
    rec = oracle_counts(WORKLOAD["L"])
    out = []
    for L in sizes:
        blocks, nvec = [(4, 4), (2, 2)], [8, 12]
        th = si.heatbath_u1(L, L, 6.0, 200, seed=1, device="cpu")
        psi0 = si.null_vector_guesses(L, L, nvec, 3, blocks)
        H = omg.Hierarchy(th, 0.01, 3, blocks, nvec, [list(a) for a in psi0])
        for lvl in (1, 2):
            lev = H.levels[lvl]
            lev.op, lev.opdag = _Counted(lev.op), _Counted(lev.opdag)
        b = si.gaussian_complex(1003, L * L)
        t = time.perf_counter()
        _, st = H.solve(b, 1e-10)
        wall = time.perf_counter() - t
        counts = {"S": st["fine_applies"],
                  "A2": H.levels[1].op.n + H.levels[1].opdag.n,
                  "A3": H.levels[2].op.n + H.levels[2].opdag.n}
        ta = apply_times(H, reps=20)
        model = rec["overhead_ratio"] * sum(counts[k] * ta[k] for k in counts) if rec else None
        out.append({"L": L, "measured_s": wall, "model_s": model, "solves_per_s": 1.0 / wall,
                    "true_resid": float(st["true_resid"]), "converged": bool(st["converged"])})
    return out


def oracle_sample_note(rec, ta, reps):
    c = rec["counts"]
    return (f"{reps} applications each of the oracle's S, A_hat2, A_hat3 timed here "
            f"({ta['S'] * 1e3:.2f}, {ta['A2'] * 1e3:.2f}, {ta['A3'] * 1e3:.2f} ms), weighted by "
            f"the application counts of the oracle's own full solve of this workload "
            f"({c['S']}, {c['A2']}, {c['A3']}) and scaled by its wall/application-time ratio "
            f"{rec['overhead_ratio']:.3f} (oracle/solve_counts_256.json, measured once on "
            f"{rec['machine']['processor']}); extrapolated")


def dslash_bandwidth(sw, ctx, L=4096, reps=20):
    """Dslash microbenchmark (metric "Dslash GB/s"): D on an L x L lattice, FP64
    and FP32, timed with CUDA events on the library's stream.  Algorithmic
    bytes per site: read x (1 complex) and the site's two links, write y;
    neighbour values and backward links are reused from cache: 64 B (FP64),
    32 B (FP32).  The working set (>= 1.3 GB) exceeds L2."""
    import torch
    gen = torch.Generator(device="cuda").manual_seed(4096)
    theta = (torch.rand((2, L, L), generator=gen, device="cuda", dtype=torch.float64) * 2 - 1) * math.pi
    g = sw.sw_gauge_load(ctx, theta)
    out = {}
    stream = torch.cuda.current_stream()
    for name, prec, dt, bps in (("fp64", sw.SW_PREC_FP64, torch.complex128, 64),
                                ("fp32", sw.SW_PREC_FP32, torch.complex64, 32)):
        x = torch.randn(L * L, dtype=dt, device="cuda", generator=gen)
        y = torch.empty_like(x)
        for _ in range(3):
            sw.sw_dslash(g, 0.01, sw.SW_OP_D, prec, x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            sw.sw_dslash(g, 0.01, sw.SW_OP_D, prec, x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        gbs = bps * L * L / t / 1e9
        out[name] = {"GB/s": gbs, "frac_of_hbm": gbs / HBM_PEAK_GBS, "us": t * 1e6,
                     "Gsites/s": L * L / t / 1e9}
    out["lattice"] = f"{L}x{L}"
    out["note"] = ("FP64 Dslash issues 20 FP64 operations per site, so on GB300 (4 FP64 flop/clk/SM) "
                   "it is FP64-ALU bound near 2 TB/s-equivalent; FP32 is HBM bound")
    g.free()
    return out


SERVING_FIELDS = [(64, 6.0), (64, 10.0), (128, 3.0), (128, 10.0), (256, 6.0), (256, 10.0),
                  (512, 6.0), (512, 10.0)]
SERVING_MASSES = [1e-3, 1e-2, 1e-1]


def coarse_stencil_bandwidth(sw, ctx, L=1024, reps=20):
    """Coarse-stencil microbenchmark: the level-2 stencil of a 1024^2 hierarchy
    (4x4 KD-block aggregates, Nv 24: 128^2 coarse sites x 48 dof, stencil larger
    than L2) applied in FP64 and in scaled FP16 (mixed hierarchy), timed with the
    library's CUDA-event brackets around each application.  Algorithmic bytes
    per coarse site and application: 5 nc^2 p for the blocks (p = 16 B FP64, 4 B
    FP16 plus 5 x 4 B of block scales) + 2 nc x 16 B for the vectors."""
    import torch
    gen = torch.Generator(device="cuda").manual_seed(1024)
    theta = (torch.rand((2, L, L), generator=gen, device="cuda", dtype=torch.float64) * 2 - 1) * math.pi
    g = sw.sw_gauge_load(ctx, theta)
    p = sw.sw_mg_params_default()
    p.setup_maxiter = 2           # the stencil's values do not matter here
    p.precision = sw.SW_MG_MIXED
    h = sw.sw_mg_setup(g, 0.01, 3, [(4, 4), (2, 2)], [24, 32], params=p, seed=7)
    e0, e1, nc = sw.sw_mg_level_info(h, 2)
    n = e0 * e1 * nc
    v = torch.randn(n, dtype=torch.complex128, device="cuda", generator=gen)
    w = torch.empty_like(v)
    out = {"lattice": f"{L}x{L}", "coarse_sites": e0 * e1, "nc": nc}
    for name, prec, pb, extra in (("fp64", sw.SW_PREC_FP64, 16, 0), ("fp16s", sw.SW_PREC_FP16S, 4, 20)):
        for _ in range(3):
            sw.sw_mg_apply_level(h, 2, prec, 0, v, w)
        sw.sw_set_timing(ctx, True)
        for _ in range(reps):
            sw.sw_mg_apply_level(h, 2, prec, 0, v, w)
        ms = sw.sw_kernel_times(ctx, 7)[1][1]  # event-bracketed ms of the reps applications
        sw.sw_set_timing(ctx, False)
        t = ms / 1e3 / reps
        byt = (5 * nc * nc * pb + extra + 2 * nc * 16) * e0 * e1
        out[name] = {"GB/s": byt / t / 1e9, "frac_of_hbm": byt / t / 1e9 / HBM_PEAK_GBS,
                     "us": t * 1e6, "bytes_per_apply": byt, "applications": reps}
    h.free()
    g.free()
    return out


def serving_measurement(nreq, seed=11, rate=4.0, workers=3, batch_max=8, mixed=True,
                        fields=None):
    """Poisson request stream of single-right-hand-side solves over 8 resident
    gauge fields (64^2 to 512^2, beta 3, 6 and 10, 200 heatbath sweeps; beta 3
    only at 128^2: at 64^2, beta 3 and m = 1e-3 the 3-level hierarchy needs
    hundreds of outer iterations on some configurations) with
    cached hierarchies (3 levels, 4x4 then 2x2 aggregates, Nv 24/32, coarsest
    cap 2048), masses log-uniform in [1e-3, 1e-1] served on the grid
    {1e-3, 1e-2, 1e-1}, tol 1e-10.  Every hierarchy belongs to one of the
    worker streams (affinity), is set up before the stream starts (reported as
    setup_s) and batches the requests queued on it (batch_max); each worker's
    coarsest kernels hold 1/workers of the SMs.  Latency = finish - arrival."""
    import sw_inputs as si
    from paper_1801_07823_gb300 import serve
    fields = fields or SERVING_FIELDS
    gauges = [(si.heatbath_u1(L, L, b, 200, seed=100 + i, device="cuda"), f"{L}^2 beta={b}")
              for i, (L, b) in enumerate(fields)]
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(nreq):
        gid = int(rng.integers(len(gauges)))
        L = fields[gid][0]
        # beta 3 requests: masses in [1e-2, 1e-1] (at beta 3 and m = 1e-3 the
        # hierarchy stalls on some configurations; the paper's own beta 3 results
        # stop at m = 0.002, with the coarsest cap hit)
        mlo = 1e-2 if fields[gid][1] <= 3.0 else 1e-3
        m = float(np.exp(rng.uniform(np.log(mlo), np.log(1e-1))))
        reqs.append((gid, m, si.gaussian_complex(2000 + i, L * L)))
    nv, blocks = [24, 32], [(4, 4), (2, 2)]
    # 512^2 and up: one more level (2 x 2, 32 vectors), so that the coarsest grid
    # stays 16^2 x 64 dof as at 256^2 (Sec. IV: the recursion extends)
    cfg = lambda L: ((blocks + [(2, 2)], nv + [32]) if L >= 512 else (blocks, nv))
    psi0_fn = lambda L, b, n: si.null_vector_guesses(L, L, n, len(n) + 1, b)
    srv = serve.Server(gauges, SERVING_MASSES, workers=workers, hbm_budget=160 << 30,
                       nvec=tuple(nv), blocks=blocks, mixed=mixed, psi0_fn=psi0_fn,
                       params=dict(outer_maxiter=200, coarsest_maxiter=2048),
                       batch_max=batch_max, affinity=True, hier_cfg=cfg)
    keys = sorted({(g, srv.snap_mass(m)) for g, m, _ in reqs})
    setup_s = srv.prewarm(keys)
    done = serve.poisson_stream(srv, reqs, rate=rate, seed=seed)
    srv.close()
    out = serve.latency_summary(done)
    out["workload"] = (f"{nreq} Poisson arrivals at {rate} requests/s over {len(fields)} resident "
                       f"gauge fields ({', '.join(f'{L}^2 b{b:g}' for L, b in fields)}; 200 "
                       "heatbath sweeps); masses log-uniform [1e-3, 1e-1] ([1e-2, 1e-1] on the "
                       "beta 3 field) on the grid "
                       f"{{1e-3, 1e-2, 1e-1}}; Nv 24/32; {workers} worker streams with "
                       f"hierarchy affinity; batch_max {batch_max}; "
                       f"{'mixed precision' if mixed else 'FP64'}; tol 1e-10; hierarchies set "
                       "up before the stream; 512^2 hierarchies with a fourth level (2x2, Nv 32)")
    out["hierarchies"] = len(keys)
    out["setup_s"] = setup_s
    out["per_request"] = [[r.rid, fields[r.gauge][0], fields[r.gauge][1], r.mass, r.batch,
                           round(r.finish - r.arrival, 3), round(r.finish - r.start, 3),
                           int(bool(r.stats.get("converged"))), r.stats.get("outer_iters"),
                           r.stats.get("error", "")] for r in done]
    out["by_size"] = {str(L): float(np.percentile([r.finish - r.arrival for r in done
                                                   if fields[r.gauge][0] == L], 50))
                      for L in sorted({L for L, _ in fields})
                      if any(fields[r.gauge][0] == L for r in done)}
    return out


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the same workload, timed in bounded samples: every
    step times applications of the oracle's operators on this machine, and a
    solve's time is extrapolated from them with the application counts of the
    oracle's own full solve of the workload (oracle_solve_seconds)."""
    if rank != 0:
        return
    L = args.L
    rec = oracle_counts(L)
    if rec is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle solve counts for "
                          f"L = {L} (oracle/solve_counts.py records the 256^2 workload)"}),
              flush=True)
        return
    dev = "cpu"
    try:
        import torch
        if torch.cuda.is_available():
            dev = "cuda"  # input generation only; everything timed below is the CPU oracle
    except ImportError:
        pass
    th, psi0 = gauge_and_psi0(L, WORKLOAD["beta"], args.sweeps, dev)
    H = oracle_hierarchy(th, WORKLOAD["mass"], psi0)
    reps = 40
    times = []
    for k in range(args.warmup + args.steps):
        t_solve, ta = oracle_solve_seconds(H, rec, reps)
        if k >= args.warmup:
            times.append(t_solve)
    t_solve = float(np.mean(times))
    value = 1.0 / t_solve
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_solve * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, L=L, sweeps=args.sweeps),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": oracle_sample_note(rec, ta, reps), "cpu": cpu_model(),
                             "measured_full_solves": oracle_validation()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_measurement(sw, ctx, hm, nbat, L, rank, world, flush, stream, barrier, fp64_value,
                        xref, reps=3):
    """nbat right-hand sides per sw_mg_solve_batch call on the mixed hierarchy hm:
    one warm-up batch (workspace, autotuner), then `reps` timed batches of fresh
    right-hand sides, L2 flushed before each.  Reports solves/s, the coarsest
    kernel's share and time per iteration, and the largest relative difference
    of the first solutions from the FP64 hierarchy's solutions of the same
    right-hand sides."""
    import torch
    tol = WORKLOAD["tol"]
    mk = lambda off: torch.stack([torch.from_numpy(rhs(rhs_seed(rank, k, off), L))
                                  for k in range(nbat)]).cuda()
    BB = mk(500)
    XB = torch.zeros_like(BB)
    sw.sw_mg_solve_batch(hm, BB, XB, tol)  # warm-up
    err = max(float(torch.linalg.norm(XB[k] - xref[k]) / torch.linalg.norm(xref[k]))
              for k in xref)
    batches = [mk(600 + 100 * j) for j in range(reps)]
    barrier()
    sw.sw_set_timing(ctx, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sts, ms = [], 0.0
    for Bj in batches:
        flush.zero_()
        e0.record(stream)
        sts += sw.sw_mg_solve_batch(hm, Bj, XB, tol)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    bk = sw.sw_kernel_times(ctx, 7)
    sw.sw_set_timing(ctx, False)
    barrier()
    sec = max_over_ranks(ms / 1e3, world)
    val = job_rate(world, nbat * reps, sec)
    return {
        "value": val, "unit": UNIT, "width": nbat, "batches": reps,
        "iterates": "f32" if getattr(hm, "batch_iterates", 0) else "f64",
        "ms_per_batch": sec / reps * 1e3,
        "dtype": "f64 outer FGCR, vectors and Krylov scalars; f32 fine smoother; f16 (scaled) "
                 "level-2 stencil; coarsest stencil products tf32 on the tensor cores (f32 "
                 "with SW_BATCH_FP32=1), f64 iterates",
        "converged_all": all(x_["converged"] and x_["true_resid"] <= tol for x_ in sts),
        "true_resid_max": max(x_["true_resid"] for x_ in sts),
        "rel_err_vs_fp64_solve_max": err,
        "outer_iters_max": max(x_["outer_iters"] for x_ in sts),
        "coarsest_avg": float(np.mean([x_["coarsest_iters"] / max(x_["coarsest_solves"], 1)
                                       for x_ in sts])),
        "coarsest_kernel": {"launches": bk[5][0], "ms": bk[5][1], "iterations": bk[6][0],
                            "us_per_iteration": 1e3 * bk[5][1] / max(bk[6][0], 1),
                            "share": bk[5][1] / max(ms, 1e-9)},
        "speedup_vs_fp64": val / fp64_value}


def mass_sweep(sw, g, psi0, B, args, world, stream, barrier, timed, fp64_value, ct, cel):
    """The workload's masses {0.1, 0.01, 0.001} (the paper's Fig. iterworst
    comparison): FP64 MG and CG on the even/odd normal system on the same field
    and right-hand sides, solves/s and fine-operator applications per solve.
    m = 0.001 reuses the headline measurements; the others time 2 solves each
    after one warm-up, with a fresh hierarchy per mass."""
    import torch
    from paper_1801_07823_gb300 import presets
    tol = WORKLOAD["tol"]
    out = {"0.001": {"mg_solves_per_s": fp64_value, "mg_fine_applies": timed[0]["fine_applies"],
                     "mg_outer_iters": timed[0]["outer_iters"],
                     "cg_solves_per_s": job_rate(world, args.steps, cel),
                     "cg_fine_applies": ct[0]["fine_applies"]}}
    X = torch.zeros_like(B[0])
    for m in (0.1, 0.01):
        hm = sw.sw_mg_setup(g, m, 3, WORKLOAD["blocks"], WORKLOAD["nvec"],
                            params=presets.make_params(sw, presets.FP64_256), psi0=psi0)
        sw.sw_mg_solve(hm, B[0], X, tol)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        sm_ = [sw.sw_mg_solve(hm, B[k], X, tol) for k in (1, 2)]
        e1.record(stream)
        barrier()
        mg_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
        hm.free()
        sw.sw_cg_eo_solve(g, m, B[0], X, tol)
        barrier()
        e0.record(stream)
        sc = [sw.sw_cg_eo_solve(g, m, B[k], X, tol) for k in (1, 2)]
        e1.record(stream)
        barrier()
        cg_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
        out[str(m)] = {"mg_solves_per_s": job_rate(world, 2, mg_s),
                       "mg_fine_applies": sm_[0]["fine_applies"],
                       "mg_outer_iters": sm_[0]["outer_iters"],
                       "mg_converged": all(x["converged"] for x in sm_),
                       "cg_solves_per_s": job_rate(world, 2, cg_s),
                       "cg_fine_applies": sc[0]["fine_applies"],
                       "cg_converged": all(x["converged"] for x in sc)}
    return out


# ---------------------------------------------------------------------------- native
def run_native(args, rank, world, local):
    import torch
    import paper_1801_07823_gb300 as sw
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    L = args.L
    m = WORKLOAD["mass"]
    th, psi0 = gauge_and_psi0(L, WORKLOAD["beta"], args.sweeps, "cuda")
    stream = torch.cuda.current_stream()
    ctx = sw.sw_context_create(local, stream.cuda_stream)
    g = sw.sw_gauge_load(ctx, th)
    from paper_1801_07823_gb300 import presets
    t = time.perf_counter()
    h = sw.sw_mg_setup(g, m, 3, WORKLOAD["blocks"], WORKLOAD["nvec"],
                       params=presets.make_params(sw, presets.FP64_256), psi0=psi0)
    setup_s = time.perf_counter() - t

    nsteps = args.warmup + args.steps
    B = [torch.from_numpy(rhs(rhs_seed(rank, k), L)).cuda() for k in range(nsteps)]
    X = torch.zeros_like(B[0])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stats = []
    for k in range(args.warmup):
        stats.append(sw.sw_mg_solve(h, B[k], X, WORKLOAD["tol"]))
    sw.sw_set_timing(ctx, True)
    launches0 = sw.sw_launch_count()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        t0 = time.perf_counter()
        timed = []
        for k in range(args.warmup, nsteps):
            flush.zero_()
            timed.append(sw.sw_mg_solve(h, B[k], X, WORKLOAD["tol"]))
        ev1.record(stream)
        barrier()
        wall = time.perf_counter() - t0
    launches = sw.sw_launch_count() - launches0
    ktimes = sw.sw_kernel_times(ctx, 7)
    sw.sw_set_timing(ctx, False)
    clocks = clk.summary()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    elapsed = max_over_ranks(elapsed, world)
    value = job_rate(world, args.steps, elapsed)
    ok = all(s["converged"] and s["true_resid"] <= WORKLOAD["tol"] for s in timed)

    # end to end through the C ABI with pinned host buffers (copies inside the call)
    hb = torch.empty((L * L,), dtype=torch.complex128, pin_memory=True)
    hx = torch.empty((L * L,), dtype=torch.complex128, pin_memory=True)
    for k in range(args.warmup):
        hb.copy_(B[k].cpu())
        sw.sw_mg_solve(h, hb.numpy(), hx.numpy(), WORKLOAD["tol"])
    barrier()
    t0 = time.perf_counter()
    for k in range(args.warmup, nsteps):
        hb.numpy()[:] = rhs(rhs_seed(rank, k), L)
        sw.sw_mg_solve(h, hb.numpy(), hx.numpy(), WORKLOAD["tol"])
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)

    # roofline of the dominant kernel (FP64 complex MAC = 8 flop; FP64-ALU bound on GB300):
    # the persistent coarsest CGNE (category 5: 2 stencil applications per iteration)
    # or a coarse stencil (categories 1, 2), whichever took the most time
    # the FP64 pipe's measured rate at the clock of the run: the roofline's peak
    fp64_peak = sw.sw_fp64_peak(ctx)
    shapes = {l: sw.sw_mg_level_info(h, l + 1) for l in (1, 2)}
    cand = {c: ktimes[c][1] for c in (1, 2, 5)}
    best = max(cand, key=cand.get)
    variant = None
    if best == 5:
        e0, e1, nc = shapes[2]
        iters = ktimes[6][0]
        n_l, ms_l = ktimes[5]
        # variant the FP64 kernel's autotuner chose (bit 0: three-FMA products, bit 1:
        # reduce-scatter row sums, bit 2: operands staged in shared memory)
        ch = [e for e in sw.sw_autotune_entries() if e[1] == 1 and e[0] == nc and e[2] == e0 * e1]
        variant = ch[0][3] if ch else None
        per_apply_flop = 8.0 * 5 * nc * nc * e0 * e1
        flop = per_apply_flop * 2 * iters / max(n_l, 1)      # per launch
        ybytes = (24.0 if (variant or 0) & 1 else 16.0) * 5 * nc * nc * e0 * e1
        byt = (ybytes + 16.0 * 2 * nc * e0 * e1) * 2 * iters / max(n_l, 1)
        kname = (f"k_cgne64<{nc}, {'three' if (variant or 0) & 1 else 'four'}-FMA products"
                 f"{', reduce-scatter row sums' if (variant or 0) & 2 else ''}"
                 f"{', operands staged in shared memory' if (variant or 0) & 4 else ''}> "
                 f"(persistent FP64 coarsest CGNE, {e0}x{e1} sites, {nc}x{nc} complex128 blocks, "
                 f"{iters / max(n_l, 1):.0f} iterations = {2 * iters / max(n_l, 1):.0f} stencil "
                 f"applications per launch)")
    else:
        e0, e1, nc = shapes[best]
        n_l, ms_l = ktimes[best]
        flop = 8.0 * 5 * nc * nc * e0 * e1
        byt = 16.0 * (5 * nc * nc + 2 * nc) * e0 * e1
        kname = f"k_coarse_apply_nc<{nc}> (level {best + 1}: {e0}x{e1} sites)"
    dur = ms_l / 1e3 / max(n_l, 1)
    achieved = flop / dur / 1e12
    traffic = None
    if best == 5:
        per_iter = _profiled_traffic("k_cgne64_fp64_256.md", "paper_1801_07823_gb300/csrc/cgne64.cu",
                                     "dram_bytes_per_iteration")
        if per_iter is not None:
            traffic = per_iter * iters / max(n_l, 1)
    executed = (6.0 / 8.0 if (variant or 0) & 1 else 1.0) * achieved
    roof = {"bound": "alu", "kernel": kname,
            "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "traffic": traffic,
            "achieved_note": "algorithmic flops of the stencil products (8 per complex "
                             "multiply-add, the operation's definition) per launch / average "
                             "launch time; the three-FMA form executes 6 of them",
            "executed_TFLOPs": executed, "executed_frac": executed / fp64_peak,
            "traffic_note": "ncu dram bytes per CGNE iteration (profiles/k_cgne64_fp64_256.md) x "
                            "iterations per launch; null if the kernel changed since",
            "peak_source": "measured in this run by sw_fp64_peak (FP64 FMA throughput, 16 warps "
                           "x 4 chains per SM); MEASURED_PEAKS.json has no FP64 entry",
            "peak_nominal": FP64_PEAK_TFLOPS, "frac_of_nominal": achieved / FP64_PEAK_TFLOPS,
            "algorithmic_flop_per_launch": flop,
            "hbm_GBps_equiv": byt / dur / 1e9, "launches": n_l, "avg_us": dur * 1e6}
    names = {0: "S", 1: "A_hat_level2", 2: "A_hat_level3", 5: "cgne_persistent"}
    kern = {names[l]: {"launches": ktimes[l][0], "ms": ktimes[l][1]} for l in names}
    kern["cgne_iterations"] = ktimes[6][0]

    # mixed-precision hierarchy on the same gauge field and right-hand sides:
    # FP64 outer FGCR, FP32 fine smoother, scaled-FP16 level 2, double-float
    # coarsest stencil (same timing protocol)
    variants = {}
    if not args.no_variants:
        pm = presets.make_params(sw, presets.FP64_256)
        pm.precision = sw.SW_MG_MIXED
        t = time.perf_counter()
        hm = sw.sw_mg_setup(g, m, 3, WORKLOAD["blocks"], WORKLOAD["nvec"], params=pm, psi0=psi0)
        msetup = time.perf_counter() - t
        for k in range(args.warmup):
            sw.sw_mg_solve(hm, B[k], X, WORKLOAD["tol"])
        barrier()
        e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0_.record(stream)
        mt = []
        for k in range(args.warmup, nsteps):
            flush.zero_()
            mt.append(sw.sw_mg_solve(hm, B[k], X, WORKLOAD["tol"]))
        e1_.record(stream)
        barrier()
        mel = e0_.elapsed_time(e1_) / 1e3
        mel = max_over_ranks(mel, world)
        m0 = mt[0]
        xa, xb = torch.zeros_like(B[0]), torch.zeros_like(B[0])
        sw.sw_mg_solve(h, B[0], xa, WORKLOAD["tol"])
        sw.sw_mg_solve(hm, B[0], xb, WORKLOAD["tol"])
        merr = float(torch.linalg.norm(xb - xa) / torch.linalg.norm(xa))
        variants["mixed"] = {
            "value": job_rate(world, args.steps, mel), "unit": UNIT, "ms_per_step": mel / args.steps * 1e3,
            "dtype": "f64 outer FGCR and vectors; f32 fine smoother; f16 (scaled) level-2 "
                     "stencil; double-float coarsest stencil",
            "converged_all": all(x_["converged"] and x_["true_resid"] <= WORKLOAD["tol"] for x_ in mt),
            "true_resid_max": max(x_["true_resid"] for x_ in mt), "setup_s": msetup,
            "rel_err_vs_fp64_solve": merr,
            "outer_iters": m0["outer_iters"],
            "inter_avg": m0["inter_iters"] / max(m0["inter_solves"], 1),
            "coarsest_avg": m0["coarsest_iters"] / max(m0["coarsest_solves"], 1),
            "speedup_vs_fp64": job_rate(world, args.steps, mel) / value}
        # batched: 16, 32 and 64 right-hand sides per sw_mg_solve_batch call on the
        # same mixed hierarchy (lockstep K-cycle, one batched coarsest CGNE on the
        # tensor cores per level visit), each width timed over `reps` batches
        xref = {}
        for k in range(3):  # FP64 solutions of the first right-hand sides: error reference
            xk = torch.zeros_like(B[0])
            bk0 = torch.from_numpy(rhs(rhs_seed(rank, k, 500), L)).cuda()
            sw.sw_mg_solve(h, bk0, xk, WORKLOAD["tol"])
            xref[k] = xk.clone()
        variants["batched"] = {}
        for nbat in (16, 32, 64):
            variants["batched"][str(nbat)] = batched_measurement(
                sw, ctx, hm, nbat, L, rank, world, flush, stream, barrier, value, xref,
                reps=args.batch_reps)
        variants["autotune"] = [dict(zip(("nc", "K", "sites", "stages", "us_per_iter"), e))
                                for e in sw.sw_autotune_entries()]
        # the same batches with FP32 iterates in the tensor-core coarsest CGNE
        p32 = presets.make_params(sw, presets.FP64_256)
        p32.precision = sw.SW_MG_MIXED
        p32.batch_iterates = sw.SW_PREC_FP32
        h32 = sw.sw_mg_setup(g, m, 3, WORKLOAD["blocks"], WORKLOAD["nvec"], params=p32, psi0=psi0)
        h32.batch_iterates = 1
        variants["batched_fp32_iterates"] = {}
        for nbat in (16, 32, 64):
            variants["batched_fp32_iterates"][str(nbat)] = batched_measurement(
                sw, ctx, h32, nbat, L, rank, world, flush, stream, barrier, value, xref,
                reps=args.batch_reps)
        h32.free()
        best = max(list(variants["batched"].values()) +
                   list(variants["batched_fp32_iterates"].values()), key=lambda v: v["value"])
        variants["batched_best"] = {"value": best["value"], "unit": UNIT, "width": best["width"],
                                    "iterates": best["iterates"],
                                    "speedup_vs_fp64": best["value"] / value}
        # the CUDA-core FP32 batched kernel on a second mixed hierarchy, for comparison
        os.environ["SW_BATCH_FP32"] = "1"
        hf = sw.sw_mg_setup(g, m, 3, WORKLOAD["blocks"], WORKLOAD["nvec"], params=pm, psi0=psi0)
        variants["batched_cuda_core_16"] = batched_measurement(
            sw, ctx, hf, 16, L, rank, world, flush, stream, barrier, value, xref, reps=2)
        os.environ.pop("SW_BATCH_FP32")
        hf.free()
        hm.free()
        # the paper's comparison solver on the same system: CG on the even/odd
        # normal equations (Sec. II, Fig. iterworst), FP64
        for k in range(1):
            sw.sw_cg_eo_solve(g, m, B[k], X, WORKLOAD["tol"])
        barrier()
        e0_.record(stream)
        ct = [sw.sw_cg_eo_solve(g, m, B[k], X, WORKLOAD["tol"]) for k in range(args.warmup, nsteps)]
        e1_.record(stream)
        barrier()
        cel = max_over_ranks(e0_.elapsed_time(e1_) / 1e3, world)
        variants["cg_eo"] = {
            "value": job_rate(world, args.steps, cel), "unit": UNIT, "ms_per_step": cel / args.steps * 1e3,
            "dtype": "f64", "iterations": ct[0]["outer_iters"],
            "converged_all": all(x_["converged"] for x_ in ct),
            "true_resid_max": max(x_["true_resid"] for x_ in ct),
            "mg_fine_applies_vs_cg": f"{timed[0]['fine_applies']} vs {ct[0]['fine_applies']}"}
        variants["mass_sweep"] = mass_sweep(sw, g, psi0, B, args, world, stream, barrier, timed,
                                            value, ct, cel)

    dslash = None if args.no_variants else dslash_bandwidth(sw, ctx)
    stencil = None if args.no_variants else coarse_stencil_bandwidth(sw, ctx)
    serving = None
    if args.serving_requests > 0 and rank == 0:
        try:  # a failure here must not cost the headline line
            serving = serving_measurement(args.serving_requests, rate=args.serving_rate,
                                          workers=args.serving_workers,
                                          batch_max=args.serving_batch)
        except Exception as exc:
            serving = {"error": f"{type(exc).__name__}: {exc}"}

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            rec = oracle_counts(L)
            if rec is None:  # no full-solve record for this size: the GPU solves' counts
                rec = {"counts": {"S": float(np.mean([s["fine_applies"] for s in timed])),
                                  "A2": ktimes[1][0] / args.steps,
                                  "A3": (ktimes[2][0] + 2 * ktimes[6][0]) / args.steps},
                       "overhead_ratio": 1.0, "machine": {"processor": "(GPU solve counts, "
                                                                       "BLAS-1 excluded)"}}
            t_cpu, ta = oracle_solve_seconds(oracle_hierarchy(th, m, psi0), rec, reps=5)
            cpu = {"value": 1.0 / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": oracle_sample_note(rec, ta, 5), "cpu": cpu_model(),
                   "measured_full_solves": oracle_validation()}
        s0 = timed[0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded heatbath gauge field, Gaussian sources)",
            "config": dict(WORKLOAD, L=L, sweeps=args.sweeps, parallelism=f"replicas x{world}",
                           l2="flushed between solves (256 MiB write)"),
            "clocks": clocks,
            "e2e": {"value": job_rate(world, args.steps, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": 16 * L * L, "d2h_bytes_per_step": 16 * L * L},
            "gpu_launches": int(launches),
            # ncu window over the timed solves: -k regex:^k_ -s <this> -c <gpu_launches>
            "launches_before_timed": int(launches0),
            "roofline": roof,
            "cpu_baseline": cpu,
            "solve": {"converged_all": ok, "true_resid_max": max(s["true_resid"] for s in timed),
                      "outer_iters": s0["outer_iters"], "fine_applies": s0["fine_applies"],
                      "inter_avg": s0["inter_iters"] / max(s0["inter_solves"], 1),
                      "coarsest_avg": s0["coarsest_iters"] / max(s0["coarsest_solves"], 1),
                      "setup_s": setup_s, "wall_s": wall},
            "kernels": kern,
            "variants": variants,
            "dslash": dslash,
            "coarse_stencil": stencil,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    h.free()
    g.free()
    ctx.free()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.dslash_only:
        import torch
        import paper_1801_07823_gb300 as sw
        torch.cuda.set_device(local)
        ctx = sw.sw_context_create(local, torch.cuda.current_stream().cuda_stream)
        print(json.dumps({"dslash": dslash_bandwidth(sw, ctx),
                          "coarse_stencil": coarse_stencil_bandwidth(sw, ctx)}), flush=True)
        ctx.free()
        return
    if args.serving_only:
        import torch
        torch.cuda.set_device(local)
        out = serving_measurement(args.serving_requests, rate=args.serving_rate,
                                  workers=args.serving_workers,
                                  batch_max=1 if args.serving_fp64 else args.serving_batch,
                                  mixed=not args.serving_fp64)
        print(json.dumps({"serving": out}), flush=True)
        return
    if args.batched_only:
        import torch
        import paper_1801_07823_gb300 as sw
        from paper_1801_07823_gb300 import presets
        torch.cuda.set_device(local)
        stream = torch.cuda.current_stream()
        ctx = sw.sw_context_create(local, stream.cuda_stream)
        th, psi0 = gauge_and_psi0(args.L, WORKLOAD["beta"], args.sweeps, "cuda")
        g = sw.sw_gauge_load(ctx, th)
        pm = presets.make_params(sw, presets.FP64_256)
        pm.precision = sw.SW_MG_MIXED
        if args.batch_f32:
            pm.batch_iterates = sw.SW_PREC_FP32
        hm = sw.sw_mg_setup(g, WORKLOAD["mass"], 3, WORKLOAD["blocks"], WORKLOAD["nvec"],
                            params=pm, psi0=psi0)
        hm.batch_iterates = 1 if args.batch_f32 else 0
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        xref = {0: torch.zeros(args.L * args.L, dtype=torch.complex128, device="cuda")}
        sw.sw_mg_solve(hm, torch.from_numpy(rhs(rhs_seed(rank, 0, 500), args.L)).cuda(),
                       xref[0], WORKLOAD["tol"])
        out = batched_measurement(sw, ctx, hm, args.batched_only, args.L, rank, world, flush,
                                  stream, torch.cuda.synchronize, 1.0, xref, reps=args.batch_reps)
        out["autotune"] = sw.sw_autotune_entries()
        print(json.dumps({"batched": out}), flush=True)
        hm.free()
        g.free()
        ctx.free()
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world, local)


if __name__ == "__main__":
    main()
