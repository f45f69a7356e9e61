"""Benchmark: unknowns*steps/s to a true relative residual of 1e-10 for the
all-at-once BDF2 system of the 1D Riesz fractional diffusion equation.

Workload (one step = one full solve, x0 = 0 -> ||F - calA U|| / ||F|| <= 1e-10):
M = 8191 interior points, Nt = 1024 time steps, kappa = 1, T = 1, alpha cycling
over {1.2, 1.5, 1.8} by step, u0 = seeded sum of 8 sine modes with N(0,1)
amplitudes, f i.i.d. N(0,1) (paper_2003_07020_gb300.workloads, "sine8_normal").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
                    [--inner strang|tau] [--impl ours|reference]

Under torchrun every rank solves its own seeded instance (independent
problems, no data-path collective; "scaling": "weak"); value = total
unknowns*steps over all ranks / max rank time.  ``--impl reference`` times
the CPU oracle (sequential BDF2 with LU) on rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M_DEF, NT_DEF, ALPHAS = 8191, 1024, (1.2, 1.5, 1.8)
ALPHAS_2D = (1.3, 1.7)
METRIC = "unknowns·steps/s to rel. residual 1e-10; mixed+learned vs plain FP64, 1 GB300"
UNIT = "unknowns*steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--inner", default=None, choices=["strang", "tau"],
                    help="Step (b) preconditioner (default: strang in 1D, tau in 2D: the 2D Strang BCCB circulant "
                         "needs up to 46 COCG iterations at 255 x 255 where the 2D tau matrix needs 7)")
    ap.add_argument("--inner-tol", type=float, default=None,
                    help="COCG relative tolerance per shifted system (library default: 1e-6 mixed, 1e-12 fp64)")
    ap.add_argument("--matvec", default="ntt", choices=["fft64", "ntt"],
                    help="1D matvec arithmetic: FP64 FFT convolution or exact NTT convolution of 58-bit rows")
    ap.add_argument("--M", type=int, default=M_DEF)
    ap.add_argument("--Nt", type=int, default=NT_DEF)
    ap.add_argument("--dim", type=int, default=1, choices=[1, 2],
                    help="2: the 2D workload (255 x 255 interior points, Nt = 256, alphas (1.3, 1.7), tau inner)")
    ap.add_argument("--batched", action="store_true",
                    help="the batched workload: 64 independent 1D instances (M in {511..4095}, Nt in {128..1024},"
                         " alpha ~ U(1.1,1.9), kappa ~ U(0.5,2)) solved together by aao_solve_batched")
    ap.add_argument("--learned", action="store_true",
                    help="the learned warm-start workload: M=1023, Nt=256, alpha ~ U(1.1,1.9); the FNO is trained "
                         "on pairs recorded from --train-instances solves, then --held-out seeds are solved "
                         "(mixed+learned, timed) and compared with plain FP64 and mixed without the model")
    ap.add_argument("--train-instances", type=int, default=2000)
    ap.add_argument("--held-out", type=int, default=200)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paper-examples", action="store_true",
                    help="Examples 1 and 2 of Sec. 4 at every size of Tables 1-6 (FP64, the paper's tau-matrix "
                         "Step (b), FGMRES / BiCGSTAB to 1e-9): Iter, TRR, Err and GPU time per row")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison arms of the default run (plain FP64, the paper's eps, config 1)")
    return ap.parse_args()


def max_over_ranks(x, world, device=None):
    """The largest x over all ranks (the job's time is its slowest rank's); x itself when world == 1.
    Works on any process-group backend (NCCL with a CUDA device, gloo on the CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # let nvidia-smi finish its NVML start-up (which can briefly stall this process's CUDA
            # calls) before the timed region: wait for its first sample, up to 5 s
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.05)
            time.sleep(0.2)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            busy = [s for s in sm if s >= 0.5 * max(sm)] or sm
            out.update(sm_mhz=statistics.median(busy), sm_max_mhz=max(smax), reasons=sorted(reasons),
                       samples=len(sm))
        return out


# ----------------------------------------------------------------------------- CPU oracle timing
def time_oracle_sample(M, Nt, alpha, n_steps, seed=0):
    """Times the oracle's sequential BDF2 (dense LU, then forward/back
    substitutions) on the first n_steps time levels.  Returns (t_lu, t_step)."""
    from oracle import fcd
    import scipy.linalg as sla
    from paper_2003_07020_gb300 import workloads
    u0, f = workloads.make_inputs(M, Nt, seed=seed)
    tau = 1.0 / Nt
    t0 = time.perf_counter()
    K = fcd.jacobian_1d(alpha, 1.0, M, 1.0 / (M + 1))
    I = np.eye(M)
    lu1 = sla.lu_factor(I - tau * K)
    lu2 = sla.lu_factor(1.5 * I - tau * K)
    t1 = time.perf_counter()
    u_prev2, u_prev1 = u0, sla.lu_solve(lu1, tau * f[0] + u0)
    for k in range(1, n_steps):
        u = sla.lu_solve(lu2, tau * f[k] + 2.0 * u_prev1 - 0.5 * u_prev2)
        u_prev2, u_prev1 = u_prev1, u
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / n_steps


def cpu_baseline(M, Nt):
    n_steps = 64
    t_lu, t_step = time_oracle_sample(M, Nt, 1.8, n_steps)
    total = t_lu + Nt * t_step
    out = {"value": M * Nt / total, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": ("sequential BDF2 (numpy/scipy FP64, dense LU) at M=%d, alpha=1.8: LU of both step "
                      "matrices %.2f s + %d of %d time steps at %.4f s each; value = M*Nt / (LU + Nt*step)"
                      % (M, t_lu, n_steps, Nt, t_step))}
    # the same sample on one core: a fresh interpreter with the BLAS thread pools limited to one thread
    import subprocess
    import sys
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench; print(json.dumps(bench.time_oracle_sample(%d, %d, 1.8, %d)))" % (M, Nt, n_steps))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600,
                           cwd=os.path.dirname(os.path.abspath(__file__)))
        t1_lu, t1_step = json.loads(r.stdout.strip().splitlines()[-1])
        out["single_core"] = {"value": M * Nt / (t1_lu + Nt * t1_step), "unit": UNIT, "cores": 1,
                              "sample": "the same sample with OMP/OpenBLAS threads = 1: LU %.2f s, step %.4f s"
                                        % (t1_lu, t1_step)}
    except Exception as e:  # the all-core figure stands on its own
        out["single_core"] = {"unavailable": "%s" % type(e).__name__}
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    M, Nt = args.M, args.Nt
    n_steps = 16
    from oracle import fcd
    import scipy.linalg as sla
    from paper_2003_07020_gb300 import workloads
    u0, f = workloads.make_inputs(M, Nt, seed=0)
    tau = 1.0 / Nt
    t0 = time.perf_counter()
    K = fcd.jacobian_1d(1.8, 1.0, M, 1.0 / (M + 1))
    lu2 = sla.lu_factor(1.5 * np.eye(M) - tau * K)
    t_lu = time.perf_counter() - t0

    def step(s):
        up2, up1 = u0, u0
        for k in range(n_steps):
            u = sla.lu_solve(lu2, tau * f[(s * n_steps + k) % Nt] + 2.0 * up1 - 0.5 * up2)
            up2, up1 = up1, u
        return u

    for s in range(args.warmup):
        step(s)
    t0 = time.perf_counter()
    for s in range(args.steps):
        step(s)
    dt = time.perf_counter() - t0
    value = M * n_steps * args.steps / dt
    sample = ("oracle sequential BDF2 time stepping (numpy/scipy FP64) at M=%d, alpha=1.8; one step = %d "
              "forward/back substitutions with the dense LU factors (factorisation %.2f s, done once "
              "before the timed steps)" % (M, n_steps, t_lu))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "1D Riesz FDE all-at-once BDF2, M=%d, Nt=%d, kappa=1" % (M, Nt), "M": M,
                       "Nt": Nt},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# FP64 and FP32 issue rates measured on GB300 by a throughput probe (DFMA and
# FFMA chains, 152 SMs): ~1.60 DFMA and ~114 FFMA per SM per 2.07 GHz clock.
FP64_PEAK_TFLOPS = 2 * 1.60 * 152 * 2.07e9 / 1e12

# DRAM bytes (read + write) per time row of matvec_f64_kernel at M = 8191 from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, 4 launches of 128 rows each, 17.02 MB per
# launch, M = 8191, Nt = 128); traffic grows with the rows, so a full launch of
# Nt rows moves Nt times this.
MATVEC_DRAM_BYTES_PER_ROW_M8191 = 17.018e6 / 128
# The same for the exact-integer (NTT) matvec of the Arnoldi steps (FP32 input, 10 of the 11 matvecs of a
# solve): ntt_quant_f32_kernel<58> + ntt_conv_kernel (4 primes) + ntt_epilogue_kernel<float, 4> (with the fused
# first CGS2 pass against 4 basis vectors) read 4.20 + 10.17 + 46.68 MB and write 0 per 128-row launch triple
# (one ncu capture at M = 8191, Nt = 128).
NTT_DRAM_BYTES_PER_ROW_M8191 = (4.200e6 + 10.171e6 + 46.684e6) / 128
# DRAM bytes of cocg_reg_kernel<Strang spectra> per shifted system at M = 8191 (13.21 MB read + 21 KB
# written for 65 systems, one ncu capture at M = 8191, Nt = 128): the per-system spectrum and tables.
COCG_DRAM_BYTES_PER_SYSTEM_M8191 = (13.211e6 + 0.021e6) / 65
# The same for cocg_tm_kernel (12.99 MB read + 6.91 MB written for 65 systems, one ncu capture at M = 8191,
# Nt = 128, profiles/cocg_tm_small_full.md): the spectrum read once and the write-back of x.
COCG_TM_DRAM_BYTES_PER_SYSTEM_M8191 = (12.988e6 + 6.912e6) / 65
# Lazy Shoup butterfly issue rate measured on GB300 (dependent-chain probe): 6.27 per clock per SM.
NTT_PEAK_GBFLY = 6.27 * 152 * 2.07


def ntt_butterflies(M, Nt):
    """Radix-2-equivalent modular butterflies of one NTT matvec: 4 primes x (forward + inverse)
    NTT of length L per time row (L/2 log2 L each)."""
    L = 4
    while L < 2 * M:
        L *= 2
    return 4 * 2 * (L // 2) * np.log2(L) * Nt
FP32_PEAK_TFLOPS = 2 * 114.0 * 152 * 2.07e9 / 1e12


def fft_flops(n):
    """Nominal flops of a complex FFT of length n (5 n log2 n)."""
    return 5.0 * n * np.log2(n)


def matvec_flops(M, Nt):
    """Algorithmic flops of one all-at-once matvec: per time row a real FFT
    convolution of length L (two complex FFTs of L/2 plus the real-signal
    split/merge and spectrum product, ~20 flops per half-length point) and
    the 5-flop BDF band."""
    L = 4
    while L < 2 * M:
        L *= 2
    return Nt * (2 * fft_flops(L // 2) + 20.0 * (L // 2) + 5.0 * M)


def cocg_flops(M, inner, inner_iters_sum, n_apply, nsys, strang_ffts=4):
    """Algorithmic flops of Step (b): per COCG iteration one Toeplitz product
    (2 complex FFTs of L) plus one preconditioner solve (tau: 2 complex FFTs of L;
    Strang: 2 with the precomputed circulant spectra of the mixed path, 4 by
    Bluestein) and ~40 flops per point of vector updates; each system also applies
    the preconditioner once before its first iteration."""
    L = 4
    while L < 2 * M:
        L *= 2
    pre = (strang_ffts if inner == "strang" else 2) * fft_flops(L)
    per_it = 2 * fft_flops(L) + pre + 40.0 * M
    return inner_iters_sum * per_it + n_apply * nsys * pre


def _pow2_at_least(x):
    L = 4
    while L < x:
        L *= 2
    return L


def matvec2d_flops(Mx, My, Nt):
    """2D matvec (Eq. 4.2 Kronecker sum): per time level, c_x T_x on the My rows and c_y T_y on the
    Mx columns, two real lines per complex FFT convolution (2 FFTs of the embedding length each),
    plus the 5-flop band and 2 adds per point."""
    Lx, Ly = _pow2_at_least(2 * Mx), _pow2_at_least(2 * My)
    rows = (My + 1) // 2 * (2 * fft_flops(Lx) + 8.0 * Lx)
    cols = (Mx + 1) // 2 * (2 * fft_flops(Ly) + 8.0 * Ly)
    return Nt * (rows + cols + 7.0 * Mx * My)


def cocg2d_flops(Mx, My, inner_iters_sum, n_apply, nsys, inner="tau"):
    """2D Step (b): per COCG iteration the Toeplitz product (My row and Mx column convolutions, 2 FFTs
    each) and the preconditioner (tau: a DST per row twice, two FFTs per column; 2D Strang: a forward and
    an inverse FFT per row, two FFTs for each of the Lx columns of the row spectra), ~50 flops per point of
    updates and dots; the preconditioner is also applied once per system before the first iteration."""
    Lx, Ly = 2 * (Mx + 1), 2 * (My + 1)
    if inner == "strang":
        pre = 2 * My * fft_flops(Lx) + 2 * Lx * fft_flops(Ly)
    else:
        pre = 2 * My * fft_flops(Lx) + 2 * Mx * fft_flops(Ly)
    per_it = 2 * My * fft_flops(Lx) + 2 * Mx * fft_flops(Ly) + pre + 50.0 * Mx * My
    return inner_iters_sum * per_it + n_apply * nsys * pre


def timed_solves(plans, Fs, reps, barrier):
    """One solve per (plan, F) pair, `reps` rounds, timed with CUDA events on the current stream after one
    untimed round; returns (ms per solve, infos of the timed solves)."""
    import torch
    U = torch.zeros(Fs[0].shape, dtype=torch.float64, device=Fs[0].device)
    for p, F in zip(plans, Fs):
        U.zero_()
        p.gmres_solve(F, U)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    barrier()
    ev0.record(stream)
    for _ in range(reps):
        for p, F in zip(plans, Fs):
            U.zero_()
            infos.append(p.gmres_solve(F, U))
    ev1.record(stream)
    barrier()
    return ev0.elapsed_time(ev1) / (reps * len(plans)), infos


def comparison_arms(args, plans, Fs, rank, dev, barrier):
    """The metric's comparison on the same config-2 inputs (and config 1): the plain FP64 solver, the mixed
    solver at the paper's circulant parameter eps = min(0.5, 0.5 tau) (Sec. 4), and the default mixed
    solver at config 1 (M = 63, Nt = 64).  Each arm: value (unknowns x steps / s), ms per solve, outer
    iterations and the largest true relative residual."""
    import torch
    from paper_2003_07020_gb300 import aao, workloads
    M, Nt = args.M, args.Nt
    out = {}

    def summary(ms, infos, m, nt):
        its = [i["outer_iters"] for i in infos]
        return {"value": m * nt / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                "outer_iters": its if len(its) <= 6 else [min(its), max(its)],
                "true_rel_res_max": max(i["true_rel_res"] for i in infos)}

    arms = [("plain_fp64", dict(prec=aao.AAO_PREC_FP64)),
            ("mixed_paper_eps", dict(prec=aao.AAO_PREC_MIXED, eps=min(0.5, 0.5 / Nt)))]
    for name, kw in arms:
        ps = [aao.Plan(M, Nt, a, kappa=1.0, T=1.0, inner=aao.AAO_INNER_STRANG,
                       matvec=aao.AAO_MATVEC_NTT if args.matvec == "ntt" else aao.AAO_MATVEC_FFT64, **kw)
              for a in ALPHAS]
        ms, infos = timed_solves(ps, Fs, 1, barrier)
        out[name] = summary(ms, infos, M, Nt)
        out[name]["eps"] = kw.get("eps", "default (min(0.5, 0.5 tau) for FP64)")
        for p in ps:
            p.close()
    # config 1: M = 63, Nt = 64, alpha 1.5, u0 = sin(pi x), f ~ U[-1, 1]
    m1, n1 = 63, 64
    p1 = aao.Plan(m1, n1, 1.5, kappa=1.0, T=1.0, prec=aao.AAO_PREC_MIXED)
    F1s = []
    for i in range(4):
        u0, f = workloads.make_inputs(m1, n1, seed=1000 * rank + i, recipe="sine1_uniform")
        F1 = torch.empty((n1, m1), dtype=torch.float64, device=dev)
        p1.build_rhs(torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev), F1)
        F1s.append(F1)
    ms, infos = timed_solves([p1] * len(F1s), F1s, 10, barrier)
    out["config1_mixed"] = summary(ms, infos, m1, n1)
    out["config1_mixed"]["workload"] = "M=63, Nt=64, alpha=1.5, kappa=1, T=1, sine1_uniform (seeds 0-3)"
    p1.close()
    return out


def run_paper_examples(args):
    """Tables 1-6 of Sec. 4 on the GPU: Example 1 by right-preconditioned FGMRES, Example 2 by preconditioned
    BiCGSTAB, each with P_eps (eps = min(0.5, 0.5 tau)) and P_1, FP64, Step (b) by the direct tau-matrix solve,
    tolerance 1e-9 from x0 = 0.  One JSON line with a row per (example, size, preconditioner): iterations,
    true relative residual, Err = max |u* - u^Nt| and the solve time (CUDA events, after one untimed solve).
    Example 2 lives on (0,2)^2 with mesh width 2/N: the library's (0,1) mesh with kappa scaled by 2^-alpha
    per direction gives the same discrete operator."""
    import torch
    from paper_2003_07020_gb300 import aao, workloads
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        info = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return info, ev0.elapsed_time(ev1)

    rows = []
    for alpha in (1.2, 1.5, 1.9):
        for Nt in (64, 256, 1024):
            for N in (128, 256, 512, 1024):
                x, u0, f = workloads.ex1_problem(alpha, Nt, N)
                ue = workloads.ex1_exact(alpha, x, 1.0)
                for name, eps in (("P_eps", min(0.5, 0.5 / Nt)), ("P_1", 1.0)):
                    with aao.Plan(N - 1, Nt, alpha, kappa=0.01, T=1.0, eps=eps, prec=aao.AAO_PREC_FP64,
                                  inner=aao.AAO_INNER_TAU_DIRECT, tol=1e-9, restart=50) as p:
                        F = torch.empty((Nt, N - 1), dtype=torch.float64, device=dev)
                        U = torch.zeros_like(F)
                        p.build_rhs(torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev), F)

                        def solve():
                            U.zero_()
                            return p.gmres_solve(F, U)
                        info, ms = timed(solve)
                        err = float(np.abs(ue - U[-1].cpu().numpy()).max())
                    rows.append({"example": 1, "alpha": alpha, "Nt": Nt, "h": "1/%d" % N, "dof": Nt * (N - 1),
                                 "precond": name, "iter": info["outer_iters"],
                                 "trr_log10": round(float(np.log10(info["true_rel_res"])), 3),
                                 "err": float("%.4e" % err), "ms": round(ms, 3)})
    for a1, a2 in ((1.4, 1.2), (1.5, 1.5), (1.7, 1.9)):
        for Nt in (64, 256, 1024):
            for N in (64, 128, 256, 512):
                X, Y, u0, f = workloads.ex2_problem(a1, a2, Nt, N)
                ue = workloads.ex2_exact(X, Y, 2.0)
                M = N - 1
                for name, eps in (("P_eps", min(0.5, 0.5 * 2.0 / Nt)), ("P_1", 1.0)):
                    with aao.Plan(M, Nt, a1, kappa=0.01 * 0.5 ** a1, T=2.0, eps=eps, My=M, alpha_y=a2,
                                  kappa_y=0.01 * 0.5 ** a2, prec=aao.AAO_PREC_FP64, inner=aao.AAO_INNER_TAU_DIRECT,
                                  tol=1e-9, restart=8, max_cycles=100) as p:
                        F = torch.empty((Nt, M, M), dtype=torch.float64, device=dev)
                        U = torch.zeros_like(F)
                        p.build_rhs(torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev), F)

                        def solve():
                            U.zero_()
                            return p.bicgstab_solve(F, U)
                        info, ms = timed(solve)
                        err = float(np.abs(ue - U[-1].cpu().numpy()).max())
                        del F, U
                    rows.append({"example": 2, "alpha": [a1, a2], "Nt": Nt, "h": "1/%d" % N, "dof": Nt * M * M,
                                 "precond": name, "iter": info["outer_iters"] / 2.0,
                                 "trr_log10": round(float(np.log10(info["true_rel_res"])), 3),
                                 "err": float("%.4e" % err), "ms": round(ms, 3)})
                del f
                torch.cuda.empty_cache()
    print(json.dumps({"mode": "paper_examples", "precision": "f64", "inner": "tau-matrix direct",
                      "rows": rows}), flush=True)


def run_ours(args):
    import torch
    from paper_2003_07020_gb300 import aao, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    M, Nt = args.M, args.Nt
    prec = aao.AAO_PREC_MIXED if args.prec == "mixed" else aao.AAO_PREC_FP64
    if args.inner is None:
        args.inner = "strang" if args.dim == 1 else "tau"
    inner = aao.AAO_INNER_STRANG if args.inner == "strang" else aao.AAO_INNER_TAU
    plans, Fs = [], []
    if args.dim == 2:
        M, My, Nt = 255, 255, 256
        p = aao.Plan(M, Nt, ALPHAS_2D[0], My=My, alpha_y=ALPHAS_2D[1], kappa=1.0, T=1.0, prec=prec, inner=inner)
        for i in range(3):
            u0, f = workloads.make_inputs_2d(M, My, Nt, seed=1000 * rank + i)
            F = torch.empty((Nt, My, M), dtype=torch.float64, device=dev)
            p.build_rhs(torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev), F)
            plans.append(p)
            Fs.append(F)
    else:
        My = 1
        for i, a in enumerate(ALPHAS):
            kw = {} if args.inner_tol is None else {"inner_tol": args.inner_tol}
            p = aao.Plan(M, Nt, a, kappa=1.0, T=1.0, prec=prec, inner=inner,
                         matvec=aao.AAO_MATVEC_NTT if args.matvec == "ntt" else aao.AAO_MATVEC_FFT64, **kw)
            u0, f = workloads.make_inputs(M, Nt, seed=1000 * rank + i)
            F = torch.empty((Nt, M), dtype=torch.float64, device=dev)
            p.build_rhs(torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev), F)
            plans.append(p)
            Fs.append(F)
    U = torch.zeros(Fs[0].shape, dtype=torch.float64, device=dev)
    infos = []

    def step(s):
        i = s % len(Fs)
        U.zero_()
        return plans[i].gmres_solve(Fs[i], U)

    for s in range(args.warmup):
        step(s)
    uniq = list({id(p): p for p in plans}.values())
    for p in uniq:
        p.get_profile(reset=True)  # launch counters run without profiling too
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        ev0.record(stream)
        for s in range(args.steps):
            infos.append(step(s))
        ev1.record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world, dev)
    launches_timed = sum(n for p in uniq for _, n in p.get_profile(reset=True).values())
    # stage breakdown: the same steps again with every launch bracketed by CUDA events (profiling
    # runs the host-driven Arnoldi steps; the timed region above replays graph-captured cycles)
    for p in uniq:
        p.set_profiling(True)
    prof_infos = [step(s) for s in range(args.steps)]
    prof = {}
    for p in uniq:
        p.set_profiling(False)
        for k, (t_ms, nl) in p.get_profile(reset=True).items():
            a, b = prof.get(k, (0.0, 0))
            prof[k] = (a + t_ms, b + nl)
    clocks = clk.summary()
    value = world * M * My * Nt * args.steps / (ms / 1e3)

    # end to end through the host-buffer entry point (pinned host memory)
    Fh = [torch.empty(Fs[0].shape, dtype=torch.float64, pin_memory=True) for _ in Fs]
    for i in range(len(Fs)):
        Fh[i].copy_(Fs[i].cpu())
    Uh = torch.empty(Fs[0].shape, dtype=torch.float64, pin_memory=True)
    barrier()
    t0 = time.perf_counter()
    for s in range(args.steps):
        plans[s % len(Fs)].gmres_solve_host(Fh[s % len(Fs)], Uh)
    barrier()
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, world, dev)
    e2e = {"value": world * M * My * Nt * args.steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": M * My * Nt * 8, "d2h_bytes_per_step": M * My * Nt * 8}

    compare = None
    if args.dim == 1 and args.prec == "mixed" and not args.no_compare:
        compare = comparison_arms(args, plans, Fs, rank, dev, barrier)
    if rank != 0:
        return
    # roofline of the dominant kernel
    pk = peaks()
    dom = max(("matvec", "cocg", "tdft_fwd", "tdft_inv", "vector"), key=lambda k: prof[k][0])
    n_apply = sum(i["outer_iters"] for i in prof_infos)
    inner_sum = sum(i["inner_iters_sum"] for i in prof_infos)
    nsys = Nt // 2 + 1
    if dom == "matvec" and args.dim == 1 and args.matvec == "ntt":
        n_mv = sum(i["matvecs"] for i in prof_infos)
        t_launch = prof["matvec"][0] / max(n_mv, 1)  # per matvec (2 kernels)
        achieved = ntt_butterflies(M, Nt) / (t_launch * 1e-3) / 1e9
        traffic = NTT_DRAM_BYTES_PER_ROW_M8191 * Nt if M == 8191 else None
        roof = {"bound": "alu", "achieved": achieved, "peak": NTT_PEAK_GBFLY, "unit": "Gbutterfly/s",
                "frac": achieved / NTT_PEAK_GBFLY, "traffic": traffic,
                "kernel": "ntt_quant_kernel + ntt_conv_kernel + ntt_epilogue_kernel",
                "peak_source": "lazy Shoup butterfly issue rate 6.27 /clk/SM x 152 SMs x 2.07 GHz (measured probe)",
                "traffic_source": "ncu dram bytes of a 128-row launch triple scaled to Nt rows" if traffic else None}
    elif dom == "matvec":
        n_mv = sum(i["matvecs"] for i in prof_infos)
        t_launch = prof["matvec"][0] / max(n_mv, 1)  # per matvec (2 kernels in 2D)
        fl = matvec_flops(M, Nt) if args.dim == 1 else matvec2d_flops(M, My, Nt)
        achieved = fl / (t_launch * 1e-3) / 1e12
        traffic = MATVEC_DRAM_BYTES_PER_ROW_M8191 * Nt if (args.dim == 1 and M == 8191) else None
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": "matvec_f64_kernel",
                "peak_source": "FP64 FMA issue rate x 152 SMs x 2.07 GHz (derived)",
                "traffic_source": "ncu dram bytes of a 128-row launch scaled to Nt rows" if traffic else None}
    elif dom == "cocg":
        t_launch = prof["cocg"][0] / max(n_apply, 1)  # per preconditioner apply
        reg = args.dim == 1 and args.prec == "mixed" and M <= 8192  # register kernel, Strang spectra
        fl = (cocg_flops(M, args.inner, inner_sum, n_apply, nsys, strang_ffts=2 if reg else 4) if args.dim == 1
              else cocg2d_flops(M, My, inner_sum, n_apply, nsys, args.inner)) / max(n_apply, 1)
        pkv = FP32_PEAK_TFLOPS if args.prec == "mixed" else FP64_PEAK_TFLOPS
        achieved = fl / (t_launch * 1e-3) / 1e12
        tm = reg and plans[0].cocg_threads == aao.AAO_COCG_TMEM  # the tensor-memory kernel
        traffic = ((COCG_TM_DRAM_BYTES_PER_SYSTEM_M8191 if tm else COCG_DRAM_BYTES_PER_SYSTEM_M8191) * nsys
                   if (reg and args.inner == "strang" and M == 8191) else None)
        roof = {"bound": "alu", "achieved": achieved, "peak": pkv, "unit": "TFLOP/s", "frac": achieved / pkv,
                "traffic": traffic,
                "kernel": ("cocg_tm_kernel" if tm else "cocg_reg_kernel") if reg else
                          ("c2d line kernels" if args.dim == 2 else "cocg_kernel"),
                "peak_source": "FMA issue rate x 152 SMs x 2.07 GHz (derived)",
                "traffic_source": "ncu dram bytes of a 65-system launch scaled to the systems" if traffic else None}
    else:
        t_launch = prof[dom][0] / max(prof[dom][1], 1)
        hb = pk.get("hbm_gbs", 6800.0)
        bytes_ = {"tdft_fwd": 16.0, "tdft_inv": 16.0, "vector": 16.0}[dom] * M * My * Nt
        achieved = bytes_ / (t_launch * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hb, "unit": "GB/s", "frac": achieved / hb,
                "traffic": None, "kernel": dom}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if args.prec == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": ("1D Riesz FDE all-at-once BDF2 to TRR<=1e-10, M=%d, Nt=%d, alpha cycling %s, "
                                "kappa=1, T=1, sine8_normal inputs" % (M, Nt, list(ALPHAS))) if args.dim == 1 else
                               ("2D Riesz FDE all-at-once BDF2 to TRR<=1e-10, %dx%d, Nt=%d, alphas %s, kappa=(1,1), "
                                "T=1, sine16_normal inputs (seeds 0-2)" % (M, My, Nt, list(ALPHAS_2D))),
                   "M": M, "My": My, "Nt": Nt, "precision": args.prec, "inner_precond": args.inner, "restart": 20,
                   "matvec": args.matvec if args.dim == 1 else "fft64",
                   "inner_tol": args.inner_tol if args.inner_tol is not None else (1e-6 if args.prec == "mixed"
                                                                                 else 1e-12),
                   "l2": "no explicit flush: every solve streams a >2 GB Krylov working set through the "
                         "129 MB L2",
                   "outer_iters": [i["outer_iters"] for i in infos],
                   "inner_iters_max": max(i["inner_iters_max"] for i in infos),
                   "true_rel_res_max": max(i["true_rel_res"] for i in infos),
                   "fgmres_cycles": "CUDA graph per restart cycle" + ("" if args.dim == 1 else
                                                                       ", COCG iterations as a WHILE node"),
                   "cocg_threads": plans[0].cocg_threads,
                   "stage_ms_profiled_pass": {k: round(v[0], 3) for k, v in prof.items()},
                   "stage_launches_profiled_pass": {k: v[1] for k, v in prof.items()}},
        "gpu_launches": int(launches_timed),
        "clocks": clocks, "roofline": roof, "e2e": e2e,
    }
    if compare:
        line["config"]["comparison"] = compare
    if world == 1 and not args.no_cpu_baseline and args.dim == 1:
        line["cpu_baseline"] = cpu_baseline(M, Nt)
    print(json.dumps(line), flush=True)
    for p in {id(p): p for p in plans}.values():
        p.close()


def fno_flops(M, B):
    """Algorithmic flops of one warm-start prediction for B systems of M points: lift (6 -> 32), per
    layer the truncated DFT and its inverse (16 modes x 32 channels, 4 flops per point each), the
    per-mode complex 32 x 32 mixes and the point-wise 32 x 32 matrix, and the projection (32 -> 2)."""
    C, K, L = 32, 16, 4
    per_layer = 2 * 4.0 * K * C * M + 8.0 * K * C * C + 2.0 * C * C * M
    return B * (2.0 * 6 * C * M + L * per_layer + 2.0 * 2 * C * M)


def run_learned(args):
    """Config of the learned warm start: train on solver-generated pairs, evaluate on held-out seeds.
    One timed step = one pass of mixed+learned solves over the held-out instances (x0 = 0 each)."""
    import torch
    from paper_2003_07020_gb300 import aao, workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    M, Nt = 1023, 256
    nsys = Nt // 2 + 1
    applies = 2
    mixed = aao.AAO_PREC_MIXED

    def setup(inst, prec):
        p = aao.Plan(M, Nt, inst["alpha"], kappa=inst["kappa"], prec=prec)
        u0, f = workloads.make_inputs(M, Nt, seed=inst["seed"])
        F = torch.empty((Nt, M), dtype=torch.float64, device=dev)
        p.build_rhs(torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev), F)
        return p, F

    # 1. training pairs recorded by the solver (first `applies` preconditioner applications of each solve)
    t0 = time.perf_counter()
    train = workloads.learned_instances(args.train_instances, seed=1 + 1000 * rank, M=M, Nt=Nt,
                                        first_seed=1_000_000 * rank)
    cap = applies * nsys * len(train)
    B_all = torch.empty((cap, M), dtype=torch.complex64, device=dev)
    X_all = torch.empty_like(B_all)
    L_all = torch.empty(cap, dtype=torch.complex128, device=dev)
    A_all = torch.empty(cap, dtype=torch.float32, device=dev)
    n = 0
    for inst in train:
        p, F = setup(inst, mixed)
        k = applies * nsys
        p.record_pairs(B_all[n:n + k], X_all[n:n + k], L_all[n:n + k])
        p.gmres_solve(F, torch.zeros_like(F))
        got = p.recorded_pairs()
        A_all[n:n + got] = inst["alpha"]
        n += got
        p.close()
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    perm = torch.randperm(n, generator=torch.Generator().manual_seed(rank)).to(dev)
    B_all, X_all = B_all[:n][perm].contiguous(), X_all[:n][perm].contiguous()
    L_all, A_all = L_all[:n][perm].contiguous(), A_all[:n][perm].contiguous()
    # 2. training (Adam, cosine learning rate from 2e-3)
    Bt = 128
    net = aao.Fno(M, max_batch=max(Bt, nsys), seed=rank)
    t0 = time.perf_counter()
    # the library's training loop (aao_fno_train): contiguous batches of the shuffled pairs, cosine schedule
    losses = list(net.train(B_all, L_all, A_all, X_all, args.train_steps, batch=Bt, lr0=2e-3, seed=0))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del B_all, X_all, L_all, A_all
    # 3. held-out instances: mixed + learned (timed), mixed without the model, plain FP64
    held = workloads.learned_instances(args.held_out, seed=2 + 1000 * rank, M=M, Nt=Nt,
                                       first_seed=1_000_000 * rank + 500_000)
    plans, Fs = [], []
    for inst in held:
        p, F = setup(inst, mixed)
        p.set_warm_start(net)
        plans.append(p)
        Fs.append(F)
    U = torch.zeros((Nt, M), dtype=torch.float64, device=dev)

    def pass_over(ps):
        out = []
        for p, F in zip(ps, Fs):
            U.zero_()
            out.append(p.gmres_solve(F, U))
        return out

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        pass_over(plans)
    for p in plans:
        p.get_profile(reset=True)
    infos = []
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            infos += pass_over(plans)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world, dev)
    launches_timed = sum(n for p in plans for _, n in p.get_profile(reset=True).values())
    cocg_threads = plans[0].cocg_threads
    for p in plans:  # stage breakdown from one more pass with every launch bracketed by events
        p.set_profiling(True)
    prof_infos = pass_over(plans)
    prof = {}
    for p in plans:
        p.set_profiling(False)
        for k, (t_ms, nl) in p.get_profile(reset=True).items():
            a, b = prof.get(k, (0.0, 0))
            prof[k] = (a + t_ms, b + nl)
    unknowns = M * Nt * len(held)
    value = world * unknowns * args.steps / (ms / 1e3)

    def timed_pass(ps):
        barrier()
        ev0.record(stream)
        inf = pass_over(ps)
        ev1.record(stream)
        barrier()
        return ev0.elapsed_time(ev1), inf

    for p in plans:
        p.set_warm_start(None)
    pass_over(plans)
    ms_cold, inf_cold = timed_pass(plans)
    # end to end (host buffers, pinned) for mixed + learned
    for p in plans:
        p.set_warm_start(net)
    Fh = [F.cpu().pin_memory() for F in Fs]  # the caller's host inputs, prepared before timing
    Uh = torch.empty((Nt, M), dtype=torch.float64, pin_memory=True)
    barrier()
    t0 = time.perf_counter()
    for p, h in zip(plans, Fh):
        p.gmres_solve_host(h, Uh)
    barrier()
    t_e2e = time.perf_counter() - t0
    del Fh
    for p in plans:
        p.close()
    plans = []
    ms_fp64, inf_fp64 = 0.0, []
    for inst, F in zip(held, Fs):
        p, _ = setup(inst, aao.AAO_PREC_FP64)
        U.zero_()
        p.gmres_solve(F, U)  # warm-up of this plan
        dt, inf = timed_pass_single(p, F, U, ev0, ev1, stream, barrier)
        ms_fp64 += dt
        inf_fp64.append(inf)
        p.close()
    if rank != 0:
        return

    def stats(inf):
        its = [i["inner_iters_sum"] / max(1, i["outer_iters"] * nsys) for i in inf]
        return {"inner_iters_per_system": round(float(np.mean(its)), 3),
                "outer_iters_mean": round(float(np.mean([i["outer_iters"] for i in inf])), 3),
                "true_rel_res_max": max(i["true_rel_res"] for i in inf)}

    pk_dom = max(("matvec", "cocg", "tdft_fwd", "tdft_inv", "vector", "fno"), key=lambda k: prof[k][0])
    n_apply = sum(i["outer_iters"] for i in prof_infos)
    if pk_dom == "fno":
        t_launch = prof["fno"][0] / max(n_apply, 1)
        achieved = fno_flops(M, nsys) / (t_launch * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "fno forward (12 kernels)",
                "peak_source": "FFMA issue rate x 152 SMs x 2.07 GHz (derived)"}
    elif pk_dom == "matvec":
        n_mv = sum(i["matvecs"] for i in prof_infos)
        t_launch = prof["matvec"][0] / max(n_mv, 1)
        achieved = matvec_flops(M, Nt) / (t_launch * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "matvec_f64_kernel",
                "peak_source": "FP64 FMA issue rate x 152 SMs x 2.07 GHz (derived)"}
    else:
        inner_sum = sum(i["inner_iters_sum"] for i in prof_infos)
        t_launch = prof["cocg"][0] / max(n_apply, 1)
        achieved = cocg_flops(M, "strang", inner_sum, n_apply, nsys) / max(n_apply, 1) / (t_launch * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "cocg_reg_kernel",
                "peak_source": "FFMA issue rate x 152 SMs x 2.07 GHz (derived)"}
    warm = stats(infos)
    warm["warm_accepted_frac"] = round(sum(i["warm_accepted"] for i in infos) /
                                       max(1, sum(i["outer_iters"] for i in infos) * nsys), 4)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32+bf16", "data": "synthetic",
            "config": {"workload": ("learned warm start: 1D M=1023, Nt=256, alpha~U(1.1,1.9), kappa=1, "
                                    "sine8_normal inputs; FNO (4 layers, width 32, 16 modes, BF16 weights) trained "
                                    "on pairs recorded from %d solver runs, evaluated on %d held-out seeds; one "
                                    "step = mixed+learned solves of all held-out instances to TRR<=1e-10"
                                    % (len(train), len(held))),
                       "M": M, "Nt": Nt, "train_pairs": n, "train_steps": args.train_steps, "batch": Bt,
                       "collect_s": round(t_collect, 2), "train_s": round(t_train, 2),
                       "loss_first": round(float(np.mean(losses[:20])), 4),
                       "loss_last": round(float(np.mean(losses[-50:])), 4),
                       "mixed_learned": warm,
                       "mixed_no_model": dict(stats(inf_cold), value=world * unknowns / (ms_cold / 1e3)),
                       "plain_fp64": dict(stats(inf_fp64), value=world * unknowns / (ms_fp64 / 1e3)),
                       "l2": "no explicit flush: each solve streams a ~100 MB Krylov basis; consecutive "
                             "instances use different plans and vectors",
                       "fgmres_cycles": "CUDA graph per restart cycle",
                       "cocg_threads": cocg_threads,
                       "stage_ms_profiled_pass": {k: round(v[0], 3) for k, v in prof.items()},
                       "stage_launches_profiled_pass": {k: v[1] for k, v in prof.items()}},
            "gpu_launches": int(launches_timed),
            "clocks": clk.summary(), "roofline": roof,
            "e2e": {"value": world * unknowns / t_e2e, "unit": UNIT,
                    "h2d_bytes_per_step": len(held) * M * Nt * 8, "d2h_bytes_per_step": len(held) * M * Nt * 8}}
    print(json.dumps(line), flush=True)
    net.close()


def timed_pass_single(p, F, U, ev0, ev1, stream, barrier):
    barrier()
    U.zero_()
    ev0.record(stream)
    inf = p.gmres_solve(F, U)
    ev1.record(stream)
    barrier()
    return ev0.elapsed_time(ev1), inf


def run_batched(args):
    """One step = one aao_solve_batched call over the 64 instances."""
    import torch
    from paper_2003_07020_gb300 import aao, workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    insts = workloads.batched_instances(64, seed=rank)
    plans, Fs, Us = [], [], []
    prec = aao.AAO_PREC_MIXED if args.prec == "mixed" else aao.AAO_PREC_FP64
    for inst in insts:
        M, Nt = inst["M"], inst["Nt"]
        p = aao.Plan(M, Nt, inst["alpha"], kappa=inst["kappa"], prec=prec)
        u0, f = workloads.make_inputs(M, Nt, seed=inst["seed"])
        F = torch.empty((Nt, M), dtype=torch.float64, device=dev)
        p.build_rhs(torch.from_numpy(u0).to(dev), torch.from_numpy(f).to(dev), F)
        plans.append(p)
        Fs.append(F)
        Us.append(torch.zeros_like(F))
    unknowns = sum(i["M"] * i["Nt"] for i in insts)

    def step():
        for U in Us:
            U.zero_()
        return aao.solve_batched(plans, Fs, Us)

    for _ in range(args.warmup):
        step()
    for p in plans:
        p.get_profile(reset=True)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    infos = []
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            infos = step()
        barrier()
        dt = time.perf_counter() - t0
    dt = max_over_ranks(dt, world, dev)
    prof_timed = {}
    for p in plans:
        for k, (_, nl) in p.get_profile(reset=True).items():
            prof_timed[k] = prof_timed.get(k, 0) + nl
    launches = sum(prof_timed.values())
    # for comparison: the concurrent-streams schedule (one host thread per instance, up to 32) ...
    for U in Us:
        U.zero_()
    aao.solve_batched(plans, Fs, Us, max_workers=32)
    barrier()
    t2 = time.perf_counter()
    for U in Us:
        U.zero_()
    aao.solve_batched(plans, Fs, Us, max_workers=32)
    barrier()
    t_streams = time.perf_counter() - t2
    # ... and the same instances solved one after another on one stream (one pass)
    for U in Us:
        U.zero_()
    barrier()
    t1 = time.perf_counter()
    for p, F, U in zip(plans, Fs, Us):
        p.gmres_solve(F, U)
    barrier()
    t_seq = time.perf_counter() - t1
    for p in plans:  # stage breakdown: one more batched step with every launch bracketed by events
        p.get_profile(reset=True)
        p.set_profiling(True)
    step()
    prof = {}
    for p in plans:
        p.set_profiling(False)
        for k, (t_ms, nl) in p.get_profile(reset=True).items():
            a, b = prof.get(k, (0.0, 0))
            prof[k] = (a + t_ms, b + nl)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": world * unknowns * args.steps / dt, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": "batched: 64 independent 1D instances, M in {511,1023,2047,4095}, Nt in "
                                   "{128,256,512,1024}, alpha~U(1.1,1.9), kappa~U(0.5,2), TRR<=1e-10 each; one step "
                                   "= one aao_solve_batched call (lockstep cycles, one Step (b) launch per Arnoldi "
                                   "step for all instances); wall-clock timing",
                       "instances": 64, "unknowns_per_step": unknowns, "precision": args.prec,
                       "step_b_launches_per_step": prof_timed.get("cocg", 0) // max(args.steps, 1),
                       "stage_launches_per_step": {k: v // max(args.steps, 1) for k, v in prof_timed.items()},
                       "concurrent_streams_ms": round(1e3 * t_streams, 2),
                       "one_by_one_ms": round(1e3 * t_seq, 2),
                       "outer_iters_max": max(i["outer_iters"] for i in infos),
                       "true_rel_res_max": max(i["true_rel_res"] for i in infos),
                       "fgmres_cycles": "lockstep host-driven steps, device Givens (the concurrent-streams and "
                                        "one-by-one comparisons replay CUDA graphs per cycle)",
                       "cocg_threads_by_M": {str(m): t for m, t in sorted({(p.M, p.cocg_threads) for p in plans})},
                       "stage_ms_sum_over_streams_profiled_step": {k: round(v[0], 3) for k, v in prof.items()}},
            "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    for p in plans:
        p.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.batched:
        run_batched(args)
    elif args.learned:
        run_learned(args)
    elif args.paper_examples:
        run_paper_examples(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
