"""Benchmark: Runge-Kutta steps of the DMFE history-integral path on GB300.

Workload (mixed (3+4)-spin, f = (q^3 + q^4)/4, T = 0.5, theta grid L = 2049 for
t_max = 1e5, stencil width 4, history store of 2049 slices, FP64): one step is one
device-driven Dormand-Prince trial step -- six stages of (history integrals, RHS
assembly), the error estimate and step rule, the append, and a sparsification pass
whenever the store is full. The state is the quench itself, solved from t = 0 until the
store has filled and been thinned once, so every timed step may run a pass.

--workload solve runs whole solves from t = 0 through checkpoints (wall clock through the
public API, truncated at --time-limit seconds and said so), optionally in several
precisions, with the differences of C, R and E between them at each checkpoint.

value: trial steps per second over all ranks (device time, CUDA events on the
solver's stream, barrier + synchronize around the timed region, max over ranks).
e2e: the same through the public C ABI from the host: per step dmfe_step(1) and a
dmfe_get_row read of the new row (device -> host), synchronised.
roofline: the history-integral kernel, timed alone with CUDA events on the same state.

--impl reference runs the FP64 CPU oracle on the same workload's shape: per step, six
whole stages of history integrals on a frozen seeded history, rows split over all host
cores.

The default run adds, at one GPU: the double-float and FP32 variants and SSPRK(10,4)
steps of the same workload; the small pure 3-spin quench end to end; the measured FP64
and FP32 FMA rates (the arithmetic roofline denominators); the kernel alone at L = 4097 in
each precision; short windows of the 256-solve batch in double-float and FP64; a batch of
small solves that all complete; the scaled serving-capacity run; the oracle on the host
cores (--no-extras skips the batch, capacity and L = 4097 parts).
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

COEFS = {3: 0.25, 4: 0.25}
T_BATH = 0.5
GRID_T_MAX = 1e5
TOL = 1e-8
# Algorithmic operations per (i, j) pair at stencil width 4, counted from the kernel
# source (FMA = 2 flops). The Lagrange weights of the three stencils are read from the
# per-grid tables, not computed per pair; the A1 and A2 weights carry the quadrature weight
# nu_i. FP64 kernel: A1 32, A2 16, B1 12 (Horner on the interval's monomial Hermite
# coefficients), B2 (stage time 2, interval coordinate 2, a 4-point stencil of 8
# coefficients 64, Horner 12), f' and f'' at two points for the (3+4) model 20, nine
# weighted products and sums 23.
FLOP_PER_PAIR_S4 = 32 + 16 + 12 + 80 + 20 + 23
# Double-float kernel, FP32 flops of the double-float arithmetic: Lagrange weights from the
# stored positions 3 x 76, B1 110, A1 220, A2 110, B2 661, f' and f'' 186, products and
# sums 205 (a renormalised double-float product 10, one left as a raw pair 7, a general sum
# 10 or 11, a sum with a small constant that is exact as a pair 4).
DF_FP32_FLOP_PER_PAIR_S4 = 228 + 110 + 220 + 110 + 661 + 186 + 205
# DRAM bytes (read + write) of one history-integral launch at this workload's state come
# from ncu captures recorded by paper_2604_06309_gb300.traffic (null once a kernel source
# has changed since its capture).
# Nominal per-GPU peaks from the unit counts and the 2.07 GHz maximum SM clock, reported
# beside the measured ones: FP64 1.25 TFLOP/s (2 FMA lanes per SM); FP32 152 SMs x 128
# lanes x 2 x 2.07e9.
FP64_NOMINAL_GFLOPS = 1250.0
FP32_NOMINAL_GFLOPS = 152 * 128 * 2 * 2.07
_ALU_PEAKS = {}
LAUNCHES_PER_STEP = 24  # step graph (begin, 6 x [prep, integrals, stage end], 4 sparsify) + begin
# Lengths of the real stability intervals (|R(-x)| <= 1 on [0, x]) of Dormand-Prince 5
# and SSPRK(10,4); with the Jacobian bound 4 sqrt(f''(1)) of Sec. 3.5 they give the
# largest stable steps.
DP5_REAL_STABILITY = 3.3066
SSPRK104_REAL_STABILITY = 13.917


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "df"])
    ap.add_argument("--L", type=int, default=2049)
    ap.add_argument("--kernel-only", action="store_true",
                    help="only launch the history-integral kernel (for profiler captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="step",
                    choices=["step", "batch", "serve", "solve", "aging", "capacity", "quench", "sparsify"],
                    help="step: the headline configuration; batch: 256 independent solves stepped "
                         "together; serve: Poisson-arrival requests with continuous batching")
    ap.add_argument("--window", type=float, default=30.0, help="seconds of batched or served work")
    ap.add_argument("--slots", type=int, default=256)
    ap.add_argument("--batch-max-L", type=int, default=4097, help="largest grid of the batch mix")
    ap.add_argument("--integrator", default="auto", choices=["auto", "dp5", "ssprk104"],
                    help="integrator of the step workload (auto: Dormand-Prince, SSPRK(10,4) after the switch)")
    ap.add_argument("--t-max", type=float, default=1e5, help="solve: final time (also the grid's t_max)")
    ap.add_argument("--checkpoints", default="1e2,1e3,1e4,1e5", help="solve: times at which to record")
    ap.add_argument("--compare", default="", help="solve: further precisions compared with --precision")
    ap.add_argument("--time-limit", type=float, default=900.0, help="solve: wall seconds per precision")
    ap.add_argument("--time-limits", default="",
                    help="solve: per-precision wall seconds, e.g. fp64:1500,df:900 (others: --time-limit)")
    ap.add_argument("--out", default="", help="solve, aging: also write the JSON result to this file")
    ap.add_argument("--serve-tmax", default="10,100", help="serve: t_max range of the requests (log-uniform)")
    ap.add_argument("--coefs", default="3:0.5", help="aging: f(q) as power:coefficient,...")
    ap.add_argument("--T", type=float, default=0.0, help="aging: bath temperature")
    ap.add_argument("--tol", type=float, default=1e-12, help="aging: RK tolerance")
    ap.add_argument("--log-r", action="store_true",
                    help="with --kernel-only, FP64: logarithmic interpolation of the response history "
                         "(App. A)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the double-float and FP32-compensated variants of the same workload")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch, capacity and L = 4097 kernel measurements of the default run")
    args = ap.parse_args()
    if args.log_r and not (args.kernel_only and args.precision == "fp64"):
        ap.error("--log-r measures the FP64 history-integral kernel: use it with --kernel-only")
    return args


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alu_peak(precision):
    """(GFLOP/s, source) of the pipe that bounds the precision's kernel: the FMA rate
    measured on this GPU by dmfe_fma_rate (FP64 for the FP64 kernel, FP32 for the
    double-float and FP32 kernels), measured once per process; nominal if that fails."""
    bits = 64 if precision == "fp64" else 32
    if bits not in _ALU_PEAKS:
        try:
            from paper_2604_06309_gb300 import fma_rate
            _ALU_PEAKS[bits] = (fma_rate(bits), "measured (dmfe_fma_rate: FMA chains, CUDA events, burst)")
        except Exception as e:  # noqa: BLE001
            _ALU_PEAKS[bits] = ((FP64_NOMINAL_GFLOPS if bits == 64 else FP32_NOMINAL_GFLOPS),
                                "nominal (measurement failed: %s)" % e)
    return _ALU_PEAKS[bits]


def traffic(precision):
    from paper_2604_06309_gb300.traffic import lookup
    return lookup(precision)


def workload(L):
    from paper_2604_06309_gb300.inputs import geometric_times
    n = L - 6
    return n, geometric_times(n, 1e-2, 9e4)


class Clocks:
    """nvidia-smi sampling (every 100 ms) around the timed region: the sampler is running
    before the region starts (the constructor waits for its first sample), and the summary
    keeps the samples whose timestamps fall inside the region that mark() and stop()
    bracket on the host clock."""

    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, idx):
        self.p = None
        self.t0 = None
        # the raw samples (the JSON line carries their summary); DMFE_CLOCKS_LOG keeps them
        self.path = os.environ.get("DMFE_CLOCKS_LOG") or os.path.join(tempfile.gettempdir(), "clocks_bench.csv")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(idx), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        deadline = time.time() + 5.0
        while time.time() < deadline and self.p.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def mark(self):
        """Host time at which the timed region starts."""
        self.t0 = time.time()

    @staticmethod
    def _stamp(x):
        from datetime import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.strptime(x, fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self):
        if self.p is None:
            return None
        t1 = time.time()
        time.sleep(0.15)  # the sample that covers the region's end
        self.p.terminate()
        self.p.wait()
        self.f.close()
        with open(self.path) as f:
            return self.summarize(f.read().splitlines(), self.t0 if self.t0 is not None else t1, t1)

    @classmethod
    def summarize(cls, lines, t0, t1):
        """Median loaded SM clock, maximum clock and active throttle reasons of the samples
        taken in [t0, t1] (host seconds; 0.1 s of slack on each side), else of the one
        nearest to the region's middle."""
        rows = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((cls._stamp(parts[0]), float(parts[1]), float(parts[2]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        inside = [r for r in rows if r[0] is not None and t0 - 0.1 <= r[0] <= t1 + 0.1]
        if not inside:
            mid = 0.5 * (t0 + t1)
            stamped = [r for r in rows if r[0] is not None]
            inside = [min(stamped, key=lambda r: abs(r[0] - mid))] if stamped else rows[-1:]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for *_, r in inside for k in range(4) if r[k].lower() == "active"})
        mx = max(r[2] for r in inside)
        loaded = [r[1] for r in inside if r[1] > 0.5 * mx] or [r[1] for r in inside]
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(inside), "region_s": round(t1 - t0, 3)}


def reduce_max_over_ranks(vals, world):
    """Each value's maximum over the ranks (an all-reduce after the timed region's barrier);
    the values themselves at N = 1."""
    if world == 1:
        return [float(x) for x in vals]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x) for x in vals], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(world, steps, max_time):
    """Steps of all ranks per second of the slowest rank (each rank runs its own replica)."""
    return world * steps / max_time


def kernel_only(sv, args, L, n0, times, rank, stream, S, flush):
    """The history-integral kernel alone on a frozen seeded history (its cost depends on
    the slice-time layout, not on the values): L - 6 slices on geometric times 1e-2 .. 9e4,
    a stage time 0.1 % beyond the last slice, L2 flushed before each launch."""
    import torch
    from paper_2604_06309_gb300.inputs import synthetic_history
    log_r = bool(getattr(args, "log_r", False))
    C, dC, R, dR = synthetic_history(20260406 + rank, times, sv.theta, sv.omega)
    sv.set_history(times, C, dC, R, dR)
    row = torch.tensor(np.concatenate([C[-1], R[-1]]), dtype=torch.float64, device="cuda")
    t_stage = float(times[-1]) * (1.0 + 1e-3)
    kt = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sv.history_integrals_dev(t_stage, row.data_ptr(), S.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            kt.append(e0.elapsed_time(e1) * 1e-3)
    torch.cuda.synchronize()
    k_avg = float(np.mean(kt))
    pairs = L * L
    hist_b = {"fp64": 64 * (n0 - 1) * L, "df": 32 * n0 * L, "fp32": 16 * n0 * L}[args.precision]
    if log_r:
        hist_b += 32 * (n0 - 1) * L   # the log-R coefficients of every interval
    tab_b = 3 * pairs * {"fp64": 40, "df": 8, "fp32": 4}[args.precision]
    hbm, src = peaks()
    per_pair = {"fp64": FLOP_PER_PAIR_S4, "df": DF_FP32_FLOP_PER_PAIR_S4}.get(args.precision)
    # (log-R mode: two exponentials per pair, no flop count stated)
    flops = pairs * per_pair if per_pair and not log_r else None
    out = {
        "metric": "history-integral launches/s", "value": 1.0 / k_avg, "unit": "launches/s",
        "n_gpus": 1, "higher_is_better": True, "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": "dmfe_history_integrals_dev on a frozen seeded history: L=%d, %d slices on "
                               "geometric times 1e-2..9e4, s=4, stage time 0.1%% beyond the last slice, "
                               "L2 flushed before each launch%s" %
                               (L, n0, ", log-R interpolation" if log_r else ""), "log_r": log_r},
        "kernel_ms": k_avg * 1e3, "algorithmic_bytes": hist_b + tab_b, "history_bytes": hist_b,
        "table_bytes": tab_b, "achieved_gbs": (hist_b + tab_b) / k_avg / 1e9,
        "hbm_frac_of_%s" % src: (hist_b + tab_b) / k_avg / 1e9 / hbm,
        "gflops": flops / k_avg / 1e9 if flops else None,
        "pair_evals_per_s": pairs / k_avg}
    if flops:
        peak, psrc = alu_peak(args.precision)
        out["alu_frac"] = {"of": "FP64" if args.precision == "fp64" else "FP32", "peak_gflops": peak,
                           "peak_source": psrc, "frac": flops / k_avg / 1e9 / peak}
    return out


def run_ours(args, rank, world):
    import torch
    from paper_2604_06309_gb300 import Solver
    from paper_2604_06309_gb300.inputs import synthetic_history

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        return _run_ours(args, rank, world, dev, stream)


def _run_ours(args, rank, world, dev, stream):
    import torch
    from paper_2604_06309_gb300 import Solver
    from paper_2604_06309_gb300.inputs import synthetic_history
    L = args.L
    n0, times = workload(L)
    log_r = bool(getattr(args, "log_r", False))
    sv = Solver(COEFS, T_BATH, L, GRID_T_MAX, s=4, history_cap=L, precision=args.precision,
                stream=stream.cuda_stream, integrator=getattr(args, "integrator", "auto"), log_r=log_r)
    S = torch.empty((10, L), dtype=torch.float64, device="cuda")
    flush = torch.empty(int(256 * 2 ** 20), dtype=torch.uint8, device="cuda")

    if args.kernel_only:
        if rank == 0:
            print(json.dumps(kernel_only(sv, args, L, n0, times, rank, stream, S, flush)))
        return None

    # ---- state: the quench solved from t = 0 until the slice store is full (steady
    # state of a capped run: every later step may trigger a sparsification pass)
    setup_steps = 0
    while True:
        sv.step(256, GRID_T_MAX, TOL, stream.cuda_stream)
        setup_steps += 256
        st0 = sv.stats()
        if st0["status"] != 0:
            raise RuntimeError("device status %d while preparing the state" % st0["status"])
        if st0["sparsify_passes"] > 0 or setup_steps >= 40000:
            break
    chunk = sv.autotune()  # work-unit size of the history-integral kernel, on this state
    t_state, Crow, Rrow, _, _ = sv.get_row()
    row = torch.tensor(np.concatenate([Crow, Rrow]), dtype=torch.float64, device="cuda")
    n_state = st0["n_slices"]
    # the kernel alone at a mid-step stage time (beyond the last slice, like stages 2..6)
    t_kernel = t_state + 0.5 * sv.stats()["dt"]

    # ---- kernel alone: history integrals on this state (L2 flushed before each launch)
    kt = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sv.history_integrals_dev(t_kernel, row.data_ptr(), S.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            kt.append(e0.elapsed_time(e1) * 1e-3)
    k_avg = float(np.mean(kt))

    # ---- device-timed steps
    sv.step(args.warmup, GRID_T_MAX, TOL, stream.cuda_stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev)
    clocks.mark()
    evs = []
    torch.cuda.nvtx.range_push("timed_steps")
    for k in range(args.steps):
        flush.zero_()  # inputs exceed L2 for FP64; the flush keeps FP32 honest too
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sv.step(1, GRID_T_MAX, TOL, stream.cuda_stream)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    dev_time = float(sum(a.elapsed_time(b) for a, b in evs) * 1e-3)
    st = sv.stats()
    if st["status"] != 0:
        raise RuntimeError("device status %d during the timed steps" % st["status"])

    # ---- end to end through the public API (host buffers, synchronous row read)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sv.step(1, GRID_T_MAX, TOL)
        sv.get_row()
    e2e_time = time.perf_counter() - t0
    st2 = sv.stats()

    pairs = L * L
    n0 = n_state
    # history read by the kernel: FP64 -- the intervals' monomial coefficients (8 doubles per
    # interval and grid point); double-float replica (4 x 8 B); FP32 replica (4 x 4 B)
    bytes_hist = {"fp64": 64 * (n0 - 1) * L, "df": 32 * n0 * L, "fp32": 16 * n0 * L}[args.precision]
    # stencil entries: {base, 4 FP64 weights} of 40 B (FP64), double-float positions of 8 B,
    # packed fixed-point positions of 4 B (FP32)
    bytes_tab = 3 * pairs * {"fp64": 40, "df": 8, "fp32": 4}[args.precision]
    bytes_io = 2 * L * 8 + 10 * L * 8
    res = dict(dev_time=dev_time, e2e_time=e2e_time, k_avg=k_avg, clocks=clk, stats=st, stats_after=st2,
               bytes=(bytes_hist, bytes_tab, bytes_io), pairs=pairs, n0=n0, t_state=t_state,
               setup_steps=setup_steps, chunk=chunk)
    sv.close()
    return res


class OracleSample:
    """The oracle on the workload's shape: the history integrals of one stage (every
    output row) on a frozen seeded history of L - 6 slices, L = the workload's grid."""

    def __init__(self, L):
        from oracle import integrals as OI
        from oracle.model import Model
        from paper_2604_06309_gb300.inputs import synthetic_history
        self.OI, self.L = OI, L
        n0, times = workload(L)
        self.G = OI.Grid(L, GRID_T_MAX, 4)
        C, dC, R, dR = synthetic_history(20260406, times, self.G.theta, self.G.omega)
        self.H = OI.History(times, C, dC, R, dR)
        self.model = Model(COEFS, T_BATH)
        self.t, self.C, self.R = float(times[-1]), C[-1], R[-1]

    def rows(self, js):
        return self.OI.history_integrals(self.model, self.G, self.H, self.t, self.C, self.R, js=js)


_ORACLE = None


def _oracle_init(L):
    global _ORACLE
    _ORACLE = OracleSample(L)


def _oracle_rows(js):
    _ORACLE.rows(js)
    return len(js)


class OraclePool:
    """Whole oracle stages on the host cores: the output rows of a stage split into blocks
    over `workers` single-threaded processes (started with spawn, before any GPU work of
    theirs; each holds its own copy of the grid and the history)."""

    def __init__(self, L, workers):
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.L, self.workers = L, workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_init, initargs=(L,))
        self.pool.map(_oracle_rows, [[0]] * workers)  # every worker has built its state

    def stages(self, n):
        """Seconds for n whole stages (every output row of each)."""
        parts = [p.tolist() for p in np.array_split(np.arange(self.L), 4 * self.workers)]
        t0 = time.perf_counter()
        for _ in range(n):
            done = sum(self.pool.map(_oracle_rows, parts))
            assert done == self.L
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(L):
    """The oracle timed on whole stages: one Dormand-Prince step (6 stages, every output
    row) on all host cores, and one stage on one core, on the workload's shape."""
    cores = host_cores()
    allc = OraclePool(L, cores)
    t_step = allc.stages(6)
    allc.close()
    one = OraclePool(L, 1)
    t_stage1 = one.stages(1)
    one.close()
    return {"value": 1.0 / t_step, "unit": "RK steps/s", "cores": cores, "kind": "oracle",
            "sample": "one whole step: 6 stages of history integrals over all %d output rows on a frozen "
                      "seeded history of %d slices (the workload's shape), rows split over %d processes "
                      "(%.1f s)" % (L, L - 6, cores, t_step),
            "one_thread": {"value": 1.0 / (6 * t_stage1), "unit": "RK steps/s", "cores": 1,
                           "sample": "one whole stage on one core (%.1f s), times 6 stages" % t_stage1}}


DTYPES = {"fp64": "f64", "fp32": "f32+f64", "df": "f32x2 (double-float)+f64"}
VARIANT_NAMES = {"fp64": "fp64", "df": "double_float", "fp32": "fp32_compensated"}


def roofline(precision, res):
    """The history-integral kernel against the resource that bounds it: the FP64 pipe (FP64
    kernel), the FP32 pipes (double-float kernel; FP32 flops of its arithmetic), HBM (FP32
    kernel). Peaks: measured on this GPU (FMA loop; MEASURED_PEAKS.json for HBM)."""
    hbm, src = peaks()
    bh, bt, bio = res["bytes"]
    k = res["k_avg"]
    pairs = res["pairs"]
    alg = bh + bt + bio
    common = {"traffic": traffic(precision), "algorithmic_bytes": alg, "history_bytes": bh, "table_bytes": bt,
              "io_bytes": bio, "hbm_frac_of_%s" % src: alg / k / 1e9 / hbm, "kernel_ms": k * 1e3}
    if precision in ("fp64", "df"):
        per_pair = FLOP_PER_PAIR_S4 if precision == "fp64" else DF_FP32_FLOP_PER_PAIR_S4
        peak, psrc = alu_peak(precision)
        ach = pairs * per_pair / k / 1e9
        out = {"kernel": "k_hi_%s (history integrals)" % ("f64" if precision == "fp64" else "df"), "bound": "alu",
               "achieved": ach, "peak": peak, "unit": "GFLOP/s", "frac": ach / peak, "peak_source": psrc,
               "flops_per_pair": per_pair,
               "nominal_peak": FP64_NOMINAL_GFLOPS if precision == "fp64" else FP32_NOMINAL_GFLOPS}
        if precision == "df":
            out["fp64_equivalent_gflops"] = pairs * FLOP_PER_PAIR_S4 / k / 1e9
        out.update(common)
        return out
    ach = alg / k / 1e9
    out = {"kernel": "k_hi_f32 (history integrals)", "bound": "hbm", "achieved": ach, "peak": hbm,
           "unit": "GB/s", "frac": ach / hbm, "peak_source": src}
    out.update(common)
    return out


def solver_info(res):
    return dict({k2: res["stats"][k2] for k2 in ("t", "steps_accepted", "steps_rejected", "sparsify_passes",
                                                 "slices_removed", "forced_removals", "n_slices", "dt",
                                                 "last_eps")},
                state_prepared_by_steps=res["setup_steps"], autotuned_unit=res["chunk"])


def run_pure3_quench():
    """The small single-instance configuration end to end: f = q^3/2, T = 0.8, L = 129,
    129-slice store, tol 1e-8, from t = 0 to 100 with one dmfe_integrate call (graph capture
    included), FP64."""
    import torch
    from paper_2604_06309_gb300 import Solver
    warm = Solver({3: 0.5}, 0.8, 129, 100.0, history_cap=129)
    warm.integrate(1.0, TOL)
    warm.close()
    torch.cuda.synchronize()
    sv = Solver({3: 0.5}, 0.8, 129, 100.0, history_cap=129)
    torch.cuda.nvtx.range_push("quench")
    t0 = time.perf_counter()
    rc = sv.integrate(100.0, TOL)
    wall = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    st = sv.stats()
    sv.close()
    steps = st["steps_accepted"] + st["steps_rejected"]
    return {"workload": "pure 3-spin f=q^3/2, T=0.8, L=129, 129-slice store, tol 1e-8, t=0..100, FP64, "
                        "one dmfe_integrate call", "status": rc, "wall_s": wall, "steps": steps,
            "rk_steps_per_s": steps / wall, "stages": st["stages"], "sparsify_passes": st["sparsify_passes"]}


# (t, t') sample points of a checkpoint tc, as multiples of tc: the last slice's row at
# sixteen ratios t'/t from 0 to 1 - 1e-4, and two-time values between stored slices
SOLVE_PAIRS = ([(1.0, r) for r in (0.0, 1e-4, 1e-3, 0.01, 0.05, 0.1, 0.2, 0.3, 0.5, 0.7, 0.8, 0.9, 0.97, 0.99,
                                   0.999, 0.9999)] +
               [(0.5, 0.25), (0.9, 0.45), (0.99, 0.5), (0.3, 0.0), (0.7, 0.69), (0.1, 0.01), (0.5, 0.49),
                (0.25, 0.2)])


def energy_threshold(coefs):
    """E_th = (f(1) - f'(1)) / sqrt(f''(1)) - f(1) sqrt(f''(1)) / f'(1) (Sec. 4.3)."""
    f = sum(coefs.values())
    f1 = sum(c * p for p, c in coefs.items())
    f2 = sum(c * p * (p - 1) for p, c in coefs.items())
    return (f - f1) / np.sqrt(f2) - f * np.sqrt(f2) / f1


def exponent_fit(t, slope, t_min=1.0):
    """Sec. 4.3: the local exponent t d/dt log(E - E_th) converges to -alpha = -2/3 for pure
    models, and its deviation is a series in t^(-1/3). Least-squares fits over t >= t_min of
    (a) slope + 2/3 = sum_{i=1..3} a_i t^(-i/3) (the paper's form, limit fixed) and
    (b) slope = -alpha + sum_{i=1..3} a_i t^(-i/3) (limit free: alpha is then an estimate)."""
    t, slope = np.asarray(t, float), np.asarray(slope, float)
    m = (t >= t_min) & np.isfinite(slope)
    if m.sum() < 6:
        return None
    tt, y = t[m], slope[m]
    basis = np.stack([tt ** (-k / 3.0) for k in (1, 2, 3)], axis=1)
    a, *_ = np.linalg.lstsq(basis, y + 2.0 / 3.0, rcond=None)
    ra = y + 2.0 / 3.0 - basis @ a
    free = np.concatenate([np.ones((len(tt), 1)), basis], axis=1)
    b, *_ = np.linalg.lstsq(free, y, rcond=None)
    rb = y - free @ b
    return {"t_range": [float(tt[0]), float(tt[-1])], "points": int(m.sum()),
            "fixed_limit": {"alpha": 2.0 / 3.0, "a": [float(x) for x in a],
                            "rms_residual": float(np.sqrt(np.mean(ra ** 2)))},
            "free_limit": {"alpha": float(-b[0]), "a": [float(x) for x in b[1:]],
                           "rms_residual": float(np.sqrt(np.mean(rb ** 2)))}}


def run_aging(args):
    """A quench to T (default the pure 3-spin f = q^3/2 to T = 0, Sec. 4.3) at a tight
    tolerance: E(t) at log-spaced times and the local exponent t d/dt log(E - E_th), which
    approaches -2/3 for pure models."""
    from paper_2604_06309_gb300 import Solver
    coefs = {int(a): float(b) for a, b in (x.split(":") for x in args.coefs.split(","))}
    eth = energy_threshold(coefs)
    sv = Solver(coefs, args.T, args.L, args.t_max, s=4, history_cap=args.L, precision=args.precision,
                integrator=args.integrator)
    times = np.exp(np.linspace(np.log(1.0), np.log(args.t_max), 81))
    rec, t0 = [], time.perf_counter()
    for tc in times:
        while True:
            sv.step(64, float(tc), args.tol)
            st = sv.stats()
            if st["status"] != 0:
                raise RuntimeError("device status %d at t = %g" % (st["status"], st["t"]))
            if st["t"] >= tc or time.perf_counter() - t0 > args.time_limit:
                break
        if st["t"] < tc:
            break
        _, _, _, mu, E = sv.get_row()
        rec.append((float(tc), E, time.perf_counter() - t0, st["steps_accepted"] + st["steps_rejected"]))
    # fluctuation-dissipation ratio X = R(t, t') / d_t' C(t, t') at the last time over the
    # aging regime t' << t (Sec. 4.4); at T = 0 it tends to x_th = sqrt(f''(1))/f'(1) -
    # 1/sqrt(f''(1)) for pure models
    tf = rec[-1][0] if rec else 0.0
    fdr = []
    if tf > 0:
        for th in (0.02, 0.05, 0.1, 0.2, 0.3):
            tp, dtp = th * tf, 1e-3 * th * tf
            cp, cm = sv.get_C([tf, tf], [tp + dtp, tp - dtp])
            r = sv.get_R([tf], [tp])[0]
            c = sv.get_C([tf], [tp])[0]
            fdr.append({"theta": th, "C": float(c), "X": float(r * 2 * dtp / (cp - cm))})
    sv.close()
    t = np.array([r[0] for r in rec])
    dE = np.array([r[1] for r in rec]) - eth
    slope = np.gradient(np.log(dE), np.log(t)) if len(t) > 2 else np.array([])
    return {"metric": "local energy exponent", "value": float(slope[-1]) if len(slope) else None,
            "exponent_fit": exponent_fit(t, slope),
            "unit": "t d log(E - E_th) / dt", "n_gpus": 1, "higher_is_better": False,
            "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": "quench of f=%s to T=%g from a random initial state, L=%d, %d-slice store, "
                                   "tol %g, integrator %s" % (args.coefs, args.T, args.L, args.L, args.tol,
                                                              args.integrator), "E_th": eth},
            "trace": [{"t": r[0], "E": r[1], "dE": float(d), "local_exponent": float(e), "wall_s": r[2],
                       "steps": r[3]} for r, d, e in zip(rec, dE, slope)],
            "fdr_at_last_time": fdr,
            "x_th_pure_T0": float(np.sqrt(sum(c * p * (p - 1) for p, c in coefs.items())) /
                                  sum(c * p for p, c in coefs.items()) -
                                  1.0 / np.sqrt(sum(c * p * (p - 1) for p, c in coefs.items())))}


def run_solve(args):
    """Whole solves of the workload from t = 0 (Secs. 3.1-3.6), recorded at checkpoints."""
    import torch
    from paper_2604_06309_gb300 import Solver
    cps = [float(x) for x in args.checkpoints.split(",") if float(x) <= args.t_max]
    precs = [args.precision] + [p for p in args.compare.split(",") if p and p != args.precision]
    limits = {a: float(b) for a, b in (x.split(":") for x in args.time_limits.split(",") if x)}
    runs = {}
    for prec in precs:
        limit = limits.get(prec, args.time_limit)
        sv = Solver(COEFS, T_BATH, args.L, args.t_max, s=4, history_cap=args.L, precision=prec,
                    integrator=args.integrator)
        t0 = time.perf_counter()
        rec, truncated = [], False
        for tc in cps:
            while True:
                sv.step(64, tc, TOL)
                st = sv.stats()
                if st["status"] != 0:
                    raise RuntimeError("%s: device status %d at t = %g" % (prec, st["status"], st["t"]))
                if st["t"] >= tc or time.perf_counter() - t0 > limit:
                    break
            wall = time.perf_counter() - t0
            if st["t"] < tc:
                truncated = True
                rec.append({"t": st["t"], "wall_s": wall, "truncated_before": tc,
                            "steps": st["steps_accepted"] + st["steps_rejected"]})
                break
            t = np.array([a * tc for a, _ in SOLVE_PAIRS])
            tp = np.array([b * tc for _, b in SOLVE_PAIRS])
            _, _, _, mu, E = sv.get_row()
            rec.append({"t": tc, "wall_s": wall, "steps": st["steps_accepted"] + st["steps_rejected"],
                        "steps_rejected": st["steps_rejected"], "stages": st["stages"],
                        "sparsify_passes": st["sparsify_passes"], "forced_removals": st["forced_removals"],
                        "dt": st["dt"], "method": "ssprk104" if st["method"] == 2 else "dp5",
                        "t_switch": st["t_switch"], "E": E, "mu": mu,
                        "C": sv.get_C(t, tp).tolist(), "R": sv.get_R(t, tp).tolist()})
            if args.out:
                # the checkpoints so far, rewritten after each one: a run that is cut off
                # still leaves them
                with open(args.out + ".partial", "w") as f:
                    json.dump(dict(runs, **{prec: {"checkpoints": rec, "time_limit_s": limit}}), f)
        runs[prec] = {"checkpoints": rec, "truncated": truncated, "time_limit_s": limit}
        sv.close()
        torch.cuda.synchronize()
    base = runs[precs[0]]["checkpoints"]
    for prec in precs[1:]:
        for a, b in zip(base, runs[prec]["checkpoints"]):
            if "C" in a and "C" in b and a["t"] == b["t"]:
                b["vs_" + precs[0]] = {"max_abs_dC": float(np.max(np.abs(np.array(a["C"]) - np.array(b["C"])))),
                                       "max_abs_dR": float(np.max(np.abs(np.array(a["R"]) - np.array(b["R"])))),
                                       "abs_dE": abs(a["E"] - b["E"])}
    last = base[-1]
    return {"metric": "RK steps/s", "value": last["steps"] / last["wall_s"], "unit": "RK steps/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": "(3+4)-spin T=0.5 quench from t=0 to %g, theta grid L=%d (t_max %g), "
                                   "%d-slice store, s=4, tol 1e-8, integrator %s; wall clock through the C ABI, "
                                   "truncated at the time limit of each precision"
                                   % (args.t_max, args.L, args.t_max, args.L, args.integrator),
                       "sample_pairs": SOLVE_PAIRS},
            "runs": runs}


BATCH_LS = (129, 257, 513, 1025, 2049, 4097)


def batch_requests(n, seed=20260406, Ls=BATCH_LS, tmax_range=(1e3, 1e6)):
    """Seeded parameter sweep: T ~ U[0.3, 1], lambda ~ U[0, 1], L = cap ~ U(Ls), t_max log-uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        T = rng.uniform(0.3, 1.0)
        lam = rng.uniform(0.0, 1.0)
        L = int(rng.choice(Ls))
        tmax = float(np.exp(rng.uniform(np.log(tmax_range[0]), np.log(tmax_range[1]))))
        out.append({"coefs": {3: 0.5 * lam, 4: 0.5 * (1.0 - lam)}, "T": T, "L": L, "t_max": tmax})
    return out


def run_sparsify(args):
    """One sparsification pass (Sec. 3.6) over a full store of L - 6 seeded slices, timed
    with CUDA events around the call (residuals, selection, compaction, the interval
    coefficients of the kept slices, and the read-back of the removed mask)."""
    import torch
    from paper_2604_06309_gb300 import Solver
    from paper_2604_06309_gb300.inputs import synthetic_history
    L = args.L
    n0, times = workload(L)
    stream = torch.cuda.Stream()
    sv = Solver(COEFS, T_BATH, L, GRID_T_MAX, s=4, history_cap=L, precision=args.precision,
                stream=stream.cuda_stream)
    C, dC, R, dR = synthetic_history(20260406, times, sv.theta, sv.omega)
    ts, removed = [], 0
    for k in range(args.warmup + args.steps):
        sv.set_history(times, C, dC, R, dR)
        sv.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mask = sv.sparsify(TOL)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            ts.append(e0.elapsed_time(e1) * 1e-3)
        removed = int(mask.sum())
    sv.close()
    avg = float(np.mean(ts))
    return {"metric": "sparsification passes/s", "value": 1.0 / avg, "unit": "passes/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": "one sparsification pass over %d seeded slices on geometric times 1e-2..9e4, "
                                   "L=%d, tol %g" % (n0, L, TOL)},
            "pass_ms": avg * 1e3, "slices_removed": removed,
            "history_bytes": 32 * n0 * L}


def run_batch(args):
    """Config 4: all requests in one batch, stepped for a fixed wall-clock window."""
    import torch
    from paper_2604_06309_gb300 import Batch, Solver
    reqs = batch_requests(args.slots, Ls=tuple(L for L in BATCH_LS if L <= args.batch_max_L))
    maxL = max(r["L"] for r in reqs)
    stream = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(stream):
        b = Batch(args.slots, maxL, maxL, precision=args.precision, stream=stream.cuda_stream)
        t0 = time.perf_counter()
        for r in reqs:
            b.add(r["coefs"], r["T"], r["L"], r["t_max"], r["t_max"], TOL, history_cap=r["L"])
        admit_s = time.perf_counter() - t0
        b.step(2)  # warm-up (graph capture, first touches)
        b.poll()
        # work-unit size of the batched kernel, tuned on this batch (one step per candidate
        # per round; the tuning steps are not timed)
        tuned, tune_ms = b.autotune(1)
        b.poll()
        st0 = [b.solver(k).stats() for k in range(len(reqs))]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
        clocks.mark()
        e0.record(stream)
        tw = time.perf_counter()
        nsteps = 0
        while time.perf_counter() - tw < args.window:
            b.step(1)
            nsteps += 1
            if nsteps % 4 == 0:
                b.poll()
        e1.record(stream)
        e1.synchronize()
        clk = clocks.stop()
        dev_s = e0.elapsed_time(e1) * 1e-3
        status, tcur, running = b.poll()
        st1 = [b.solver(k).stats() for k in range(len(reqs))]
        stages = sum(a["stages"] - z["stages"] for a, z in zip(st1, st0))
        pairs = sum((a["stages"] - z["stages"]) * r["L"] ** 2 for a, z, r in zip(st1, st0, reqs))
        completed = int(sum(1 for x in status[:len(reqs)] if x == 1))
        failed = int(sum(1 for x in status[:len(reqs)] if -100 < x < 0))
        res = {"batched_steps": nsteps, "device_s": dev_s, "instance_stages_per_s": stages / dev_s,
               "pair_evals_per_s": pairs / dev_s, "completed": completed, "failed": failed,
               "completed_solves_per_s": completed / dev_s, "admission_s": admit_s, "clocks": clk,
               "tuned_unit": tuned, "tune_ms_per_step": {str(k): v for k, v in tune_ms.items()},
               "max_t_reached": float(np.max(tcur[:len(reqs)]))}
        b.close()
        # one at a time on the same GPU, FP64: stage time of a single solve per grid size
        single = {}
        for L in sorted(set(r["L"] for r in reqs)):
            sv = Solver(MIX_FOR_SINGLE, 0.5, L, 1e5, history_cap=L, precision="fp64", stream=stream.cuda_stream)
            sv.step(3, 1e5, TOL, stream.cuda_stream)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            sv.step(8, 1e5, TOL, stream.cuda_stream)
            a1.record(stream)
            a1.synchronize()
            single[L] = a0.elapsed_time(a1) * 1e-3 / (8 * 6)
            sv.close()
        t_single = sum(single[r["L"]] for r in reqs)          # seconds for one stage of every solve
        res["single_fp64_instance_stages_per_s"] = len(reqs) / t_single
        res["gain_vs_single_fp64"] = res["instance_stages_per_s"] / res["single_fp64_instance_stages_per_s"]
        res["single_fp64_stage_ms"] = {str(L): 1e3 * v for L, v in single.items()}
    return res


def run_batch_complete(args, precision, n_req=64, Ls=(129, 257), tmax_range=(1e2, 1e3), seed=20260406,
                       window=90.0, single_window=30.0):
    """Completed solves/s of a batch (config 4's mix of T and lambda on small grids with
    t_max log-uniform in [1e2, 1e3], so that every member finishes): all n_req solves admitted
    at once into one batch and stepped until each reaches its t_max; against the same
    requests solved one at a time by the plain FP64 solver (one dmfe_integrate each, for a
    fixed wall window), with E compared on every request finished by both."""
    import torch
    from paper_2604_06309_gb300 import Batch, Solver
    reqs = batch_requests(n_req, seed=seed + 3, Ls=Ls, tmax_range=tmax_range)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = Batch(n_req, max(Ls), max(Ls), precision=precision, stream=stream.cuda_stream)
        for r in reqs:
            b.add(r["coefs"], r["T"], r["L"], r["t_max"], r["t_max"], TOL, history_cap=r["L"])
        t0 = time.perf_counter()
        running = n_req
        while running > 0 and time.perf_counter() - t0 < window:
            b.step(16)
            status, _, running = b.poll()
        wall = time.perf_counter() - t0
        status, tcur, running = b.poll()
        E = {}
        for k in range(n_req):
            if status[k] == 1:
                E[k] = b.solver(k).get_row()[4]
        b.close()
    done = len(E)
    seq, t1 = {}, time.perf_counter()
    for k, r in enumerate(reqs):
        if time.perf_counter() - t1 > single_window:
            break
        sv = Solver(r["coefs"], r["T"], r["L"], r["t_max"], history_cap=r["L"], precision="fp64")
        if sv.integrate(r["t_max"], TOL) == 0:
            seq[k] = sv.get_row()[4]
        sv.close()
    seq_wall = time.perf_counter() - t1
    both = [k for k in seq if k in E]
    rate, seq_rate = done / wall, len(seq) / seq_wall
    return {"workload": "%d solves, T~U[0.3,1], lambda~U[0,1], L=cap~U{%s}, t_max~logU[%g,%g], tol 1e-8, "
                        "one batch stepped until all finish" % (n_req, ",".join(map(str, Ls)), *tmax_range),
            "precision": precision, "completed": done, "failed": int(sum(1 for x in status[:n_req] if -100 < x < 0)),
            "wall_s": wall, "completed_solves_per_s": rate,
            "single_fp64_completed": len(seq), "single_fp64_wall_s": seq_wall,
            "single_fp64_solves_per_s": seq_rate, "gain_vs_single_fp64": rate / seq_rate if seq_rate else None,
            "requests_compared": len(both),
            "max_abs_dE_vs_single_fp64": max((abs(E[k] - seq[k]) for k in both), default=None)}


def run_capacity(args, n_req=256, seed=20260406):
    """Solves/s of the serving loop when it is never idle: n_req requests of the scaled
    serving mix (L~U{65,129,257}, t_max~logU[10,100]) are all queued at once and served
    with continuous batching; against the same requests solved one at a time by the plain
    FP64 solver (each solve one dmfe_integrate call, for a fixed wall window). E of every
    request finished by both is compared."""
    import torch
    from paper_2604_06309_gb300 import Server, Solver
    reqs = batch_requests(n_req, seed=seed + 2, Ls=SERVE_LS, tmax_range=(10.0, 100.0))
    free, _ = torch.cuda.mem_get_info()
    srv = Server(args.slots, max(SERVE_LS), max(SERVE_LS), precision=args.precision, hbm_budget=int(0.5 * free),
                 steps_per_round=4)
    t0 = time.perf_counter()
    ids = [srv.submit(r["coefs"], r["T"], r["L"], r["t_max"], r["t_max"], TOL, history_cap=r["L"]) for r in reqs]
    results = []
    while len(results) < n_req and time.perf_counter() - t0 < args.window:
        results += srv.poll()
        time.sleep(0.005)
    wall = time.perf_counter() - t0
    results += srv.poll()
    srv.stop()
    ok = {r["id"]: r for r in results if r["status"] == 0}
    served_rate = len(ok) / wall
    # the same requests one at a time, FP64, one dmfe_integrate per solve
    seq, t1 = {}, time.perf_counter()
    for rid, r in zip(ids, reqs):
        if time.perf_counter() - t1 > args.window:
            break
        sv = Solver(r["coefs"], r["T"], r["L"], r["t_max"], history_cap=r["L"], precision="fp64")
        if sv.integrate(r["t_max"], TOL) == 0:
            seq[rid] = sv.get_row()[4]
        sv.close()
    seq_wall = time.perf_counter() - t1
    seq_rate = len(seq) / seq_wall
    both = [rid for rid in seq if rid in ok]
    dE = max(abs(ok[rid]["E"] - seq[rid]) for rid in both) if both else None
    lat = np.array([r["done_s"] - r["submit_s"] for r in ok.values()]) if ok else np.array([np.nan])
    return {"metric": "served solves/s (saturated)", "value": served_rate, "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": "%d requests of (3+4)-spin solves, T~U[0.3,1], lambda~U[0,1], L=cap~U{65,129,257}, "
                                   "t_max~logU[10,100], tol 1e-8, all queued at t=0, continuous batching in %d slots"
                                   % (n_req, args.slots), "window_s": args.window},
            "capacity": {"completed": len(ok), "wall_s": wall, "p50_latency_s": float(np.median(lat)),
                         "p99_latency_s": float(np.percentile(lat, 99)),
                         "single_fp64_completed": len(seq), "single_fp64_wall_s": seq_wall,
                         "single_fp64_solves_per_s": seq_rate, "gain_vs_single_fp64": served_rate / seq_rate,
                         "requests_compared": len(both), "max_abs_dE_vs_single_fp64": dE}}


MIX_FOR_SINGLE = {3: 0.25, 4: 0.25}
SERVE_LS = (65, 129, 257)


def run_serving(args, rate=20.0, seed=20260406):
    """Poisson arrivals of (3+4)-spin requests (T~U[0.3,1], lambda~U[0,1], L~U{65,129,257},
    t_max log-uniform in --serve-tmax), admitted by device footprint into a continuously
    stepped batch. The default t_max range [10, 100] reaches a steady state within a
    minute; the configuration's own range [1e3, 1e7] does not (the queue grows), and its
    run reports admissions, completions and the queue over the window."""
    import torch
    from paper_2604_06309_gb300 import Server, footprint
    rng = np.random.default_rng(seed)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    srv = Server(args.slots, max(SERVE_LS), max(SERVE_LS), precision=args.precision, hbm_budget=budget,
                 steps_per_round=4)
    tr = tuple(float(x) for x in args.serve_tmax.split(","))
    reqs = batch_requests(100000, seed=seed + 1, Ls=SERVE_LS, tmax_range=tr)
    t0 = time.perf_counter()
    next_arrival = rng.exponential(1.0 / rate)
    submitted, results, peak_bytes, samples = 0, [], 0, []
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.mark()
    while True:
        now = time.perf_counter() - t0
        if now >= args.window:
            break
        while next_arrival <= now and submitted < len(reqs):
            r = reqs[submitted]
            srv.submit(r["coefs"], r["T"], r["L"], r["t_max"], r["t_max"], TOL, history_cap=r["L"])
            submitted += 1
            next_arrival += rng.exponential(1.0 / rate)
        results += srv.poll()
        st = srv.stats()
        peak_bytes = max(peak_bytes, st["bytes_in_use"])
        samples.append((now, st["running"], st["queued"]))
        time.sleep(0.002)
    clk = clocks.stop()
    st = srv.stats()
    results += srv.poll()
    srv.stop()
    ok = [r for r in results if r["status"] == 0]
    lat = np.array([r["done_s"] - r["submit_s"] for r in ok]) if ok else np.array([np.nan])
    wait = np.array([r["admit_s"] - r["submit_s"] for r in ok]) if ok else np.array([np.nan])
    second_half = [r for r in ok if r["done_s"] > args.window / 2]
    return {"metric": "served solves/s", "value": len(ok) / args.window, "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": "Poisson arrivals %.0f req/s of (3+4)-spin solves, T~U[0.3,1], lambda~U[0,1], "
                                   "L=cap~U{%s}, t_max~logU[%g,%g], tol 1e-8, seed %d, continuous batching"
                                   % (rate, ",".join(map(str, SERVE_LS)), tr[0], tr[1], seed),
                       "window_s": args.window, "max_slots": args.slots, "hbm_budget_bytes": budget},
            "serve": {"submitted": submitted, "completed": len(ok), "failed": st["failed"],
                      "queued_at_end": st["queued"], "running_at_end": st["running"],
                      "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
                      "p50_queue_wait_s": float(np.percentile(wait, 50)),
                      "solves_per_s_second_half": len(second_half) / (args.window / 2),
                      "mean_running": float(np.mean([x[1] for x in samples])) if samples else 0.0,
                      "peak_hbm_bytes": peak_bytes, "hbm_utilisation_of_total": peak_bytes / total,
                      "batched_steps": st["batched_steps"], "admitted": st["admitted"],
                      "queue_over_time": [(round(x[0], 1), x[1], x[2]) for x in
                                          samples[::max(1, len(samples) // 10)]],
                      "completed_t_max_max": max((r["t_final"] for r in ok), default=0.0),
                      "failed_status_counts": {str(c): sum(1 for r in results if r["status"] == c)
                                               for c in sorted({r["status"] for r in results if r["status"] != 0})}},
            "clocks": clk}


def run_extras(args, rank):
    """The default run's further measurements (one GPU): each guarded, so that one failure
    is reported in the line instead of losing the headline."""
    import torch
    out = {}

    def guarded(key, fn):
        try:
            out[key] = fn()
        except Exception as e:  # noqa: BLE001
            out[key] = {"error": "%s: %s" % (type(e).__name__, e)}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    def k4097():
        from paper_2604_06309_gb300 import Solver
        res = {}
        L = 4097
        n0, times = workload(L)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            S = torch.empty((10, L), dtype=torch.float64, device="cuda")
            flush = torch.empty(int(256 * 2 ** 20), dtype=torch.uint8, device="cuda")
            for prec in ("fp64", "df", "fp32"):
                a2 = argparse.Namespace(**vars(args))
                a2.precision, a2.log_r = prec, False
                sv = Solver(COEFS, T_BATH, L, GRID_T_MAX, s=4, history_cap=L, precision=prec,
                            stream=stream.cuda_stream)
                r = kernel_only(sv, a2, L, n0, times, rank, stream, S, flush)
                sv.close()
                res[VARIANT_NAMES[prec]] = {k: r[k] for k in ("kernel_ms", "pair_evals_per_s", "algorithmic_bytes",
                                                            "history_bytes", "table_bytes", "achieved_gbs",
                                                            "gflops") if k in r}
                res[VARIANT_NAMES[prec]].update({k: v for k, v in r.items() if k.startswith("hbm_frac")
                                                 or k == "alu_frac"})
        return res

    def batch(prec, window):
        a2 = argparse.Namespace(**vars(args))
        a2.precision, a2.window = prec, window
        r = run_batch(a2)
        r.pop("clocks", None)
        return r

    guarded("kernel_only_L4097", k4097)
    guarded("batch_config4_double_float", lambda: batch("df", 10.0))
    guarded("batch_config4_fp64", lambda: batch("fp64", 10.0))
    guarded("batch_completing_double_float", lambda: run_batch_complete(args, "df"))

    def capacity():
        a2 = argparse.Namespace(**vars(args))
        a2.precision, a2.window = "df", 30.0
        return run_capacity(a2)["capacity"]

    guarded("capacity_double_float", capacity)
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cfg = {"workload": "mixed (3+4)-spin T=0.5 quench, theta grid L=%d (t_max 1e5), %d-slice store, s=4"
                       % (args.L, args.L),
           "f": "(q^3+q^4)/4", "T": T_BATH, "L": args.L, "history_cap": args.L, "s": 4, "tol": TOL,
           "replicas": world, "l2": "flushed before every timed step (256 MB write)"}
    if args.impl == "reference":
        if rank != 0:
            return
        cores = host_cores()
        pool = OraclePool(args.L, cores)
        steps_t = [pool.stages(6) for _ in range(args.warmup + args.steps)]
        pool.close()
        v = 1.0 / float(np.mean(steps_t[args.warmup:]))
        line = {"impl": "reference", "metric": "RK steps/s", "value": v, "unit": "RK steps/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": v, "unit": "RK steps/s", "cores": cores, "kind": "oracle",
                                 "sample": "per step: 6 whole stages of history integrals (all %d output rows) on "
                                           "a frozen seeded history of %d slices, rows split over %d processes"
                                           % (args.L, args.L - 6, cores)},
                "e2e": {"value": v, "unit": "RK steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.workload == "sparsify":
        print(json.dumps(run_sparsify(args)))
        return
    if args.workload == "batch":
        r = run_batch(args)
        line = {"metric": "instance-stages/s", "value": r["instance_stages_per_s"], "unit": "instance-stages/s",
                "n_gpus": 1, "higher_is_better": True, "dtype": DTYPES[args.precision], "data": "synthetic",
                "config": {"workload": "%d independent (3+4)-spin solves, T~U[0.3,1], lambda~U[0,1], L=cap~U{%s}, "
                                       "t_max~logU[1e3,1e6], tol 1e-8, seed 20260406, one persistent launch per "
                                       "stage, graph per batched step" % (args.slots, ",".join(map(str, BATCH_LS))),
                           "window_s": args.window},
                "batch": r}
        print(json.dumps(line))
        return
    if args.workload == "serve":
        print(json.dumps(run_serving(args)))
        return
    if args.workload in ("solve", "aging"):
        r = run_solve(args) if args.workload == "solve" else run_aging(args)
        if args.out:
            with open(args.out, "w") as f:
                json.dump(r, f)
        print(json.dumps(r))
        return
    if args.workload == "capacity":
        print(json.dumps(run_capacity(args)))
        return
    if args.workload == "quench":
        q = run_pure3_quench()
        print(json.dumps({"metric": "RK steps/s", "value": q["rk_steps_per_s"], "unit": "RK steps/s", "n_gpus": 1,
                          "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": q["workload"]}, "quench": q}))
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    res = run_ours(args, rank, world)
    if res is None:
        return
    dev_time, e2e_time = reduce_max_over_ranks([res["dev_time"], res["e2e_time"]], world)
    if rank != 0:
        return
    value = whole_job_rate(world, args.steps, dev_time)
    L = args.L
    roof = roofline(args.precision, res)
    line = {"metric": "RK steps/s", "value": value, "unit": "RK steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_time / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision],
            "data": "synthetic", "config": cfg,
            "e2e": {"value": whole_job_rate(world, args.steps, e2e_time), "unit": "RK steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 2 * L * 8 + 3 * 8},
            "gpu_launches": args.steps * LAUNCHES_PER_STEP,
            "roofline": roof, "clocks": res["clocks"], "solver": solver_info(res)}
    if not args.no_variants and world == 1:
        variants = {}
        for prec in ("df", "fp32", "fp64"):
            if prec == args.precision:
                continue
            a2 = argparse.Namespace(**vars(args))
            a2.precision = prec
            r2 = run_ours(a2, rank, world)
            variants[VARIANT_NAMES[prec]] = {
                "value": args.steps / r2["dev_time"], "e2e": args.steps / r2["e2e_time"], "unit": "RK steps/s",
                "dtype": DTYPES[prec], "roofline": roofline(prec, r2), "solver": solver_info(r2)}
        # the late-time integrator on the same workload: ten stages per step, a real
        # stability interval of 13.9 instead of 3.31 (Sec. 3.5)
        a3 = argparse.Namespace(**vars(args))
        a3.integrator = "ssprk104"
        r3 = run_ours(a3, rank, world)
        ssp = args.steps / r3["dev_time"]
        rho = 4.0 * np.sqrt(sum(c * p * (p - 1) for p, c in COEFS.items()))
        variants["ssprk104_" + VARIANT_NAMES[args.precision]] = {
            "value": ssp, "e2e": args.steps / r3["e2e_time"], "unit": "RK steps/s", "dtype": DTYPES[args.precision],
            "stage_evals_per_s": 10 * ssp, "gpu_launches_per_step": 35,
            "simulated_time_per_s_at_stability_limit": ssp * SSPRK104_REAL_STABILITY / rho,
            "dp5_simulated_time_per_s_at_stability_limit": value * DP5_REAL_STABILITY / rho,
            "roofline": roofline(args.precision, r3), "solver": solver_info(r3)}
        line["variants"] = variants
    if not args.no_variants and world == 1:
        line["pure3_quench"] = run_pure3_quench()
    if not args.no_extras and world == 1:
        line["alu_peaks_gflops"] = {"fp64": alu_peak("fp64")[0], "fp32": alu_peak("fp32")[0],
                                    "source": alu_peak("fp64")[1]}
        line["extras"] = run_extras(args, rank)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(L)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
