"""Benchmark: randomized SVD solves/s on one GB300 (or N replicas).

Default workload: the polynomial-decay matrix A = U diag(j^-1.5) V^T, 32768 x
32768 float32 with Haar U, V (4.29 GB, far larger than the 129 MB L2), rank
k = 200 with p = 56 (l = 256) and q = 2 power steps, bf16 sketches.  One step
= one full rsvd_fixed_rank call (every row of the path: Omega, the six
tensor-core passes over A, CholeskyQR2 after each product, B^T = A^T Q in
split bf16, the small SVD, the lift to U and V).

``--workload pca``: the 2^20 x 4096 PCA-shaped matrix (rank-64 signal plus
noise, column-centred), k = 64, p = 64, q = 1, e4m3 sketches with one scale
per 128-row block of A.

``--workload batched``: 4096 kernel-matrix blocks (1 / |x_i - y_j| between two
point clouds 3 apart, m, n ~ U{64..1024}) solved to relative Frobenius
tolerance 1e-6 by rsvd_batched, one persistent launch replayed from a CUDA
graph; one step = the whole batch, `value` = blocks solved per second.

``--workload controller``: a stream of square matrices solved to tolerance
1e-4 with the learned (l, q) controller (trained first, on the GPU).

``--workload nystrom``: the Nystrom EVD (Fig. nystrom) of a 16384^2 SPD
matrix V diag(j^-1.5) V^T in binary32, beside the fixed-rank RSVD with the
same passes over A.

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
matrix (replicas; there is no exchange step), and `value` is the total over
ranks.  ``--impl reference`` times the float64 CPU oracle instead, on a
bounded sample of the same workload: rsvd_power on a smaller matrix of the
same family (poly, pca), nystrom on a smaller SPD matrix, adaptive_blocked on
the first blocks of the batch, and adaptive_blocked on size-capped stand-ins
of the controller stream's matrices, each scaled to the full size by m n.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RSVD solves/s and % roofline at stated FP64-oracle error; mixed vs plain FP32"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poly", choices=["poly", "pca", "controller", "batched", "nystrom"],
                    help="poly: 32768^2 polynomial decay (bf16); pca: 2^20 x 4096 PCA matrix (e4m3); "
                         "controller: a stream of square matrices solved to tol 1e-4 (learned controller); "
                         "batched: 4096 kernel-matrix blocks to tol 1e-6 in one persistent launch")
    ap.add_argument("--count", type=int, default=4096, help="batched: number of blocks")
    ap.add_argument("--train", type=int, default=192, help="controller: training matrices")
    ap.add_argument("--lo", type=int, default=512, help="controller: smallest n")
    ap.add_argument("--hi", type=int, default=16384, help="controller: largest n")
    ap.add_argument("--prec", default=None, choices=["bf16", "f32", "fp8", "fp8b"],
                    help="fp8: e4m3 with a scale per row; fp8b: one scale per 128-row block")
    ap.add_argument("--m", type=int, default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--p", type=int, default=None)
    ap.add_argument("--q", type=int, default=None)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-f32", action="store_true")
    ap.add_argument("--sample", type=int, default=None, help="CPU oracle sample size (rows; square for poly)")
    ap.add_argument("--cpu-sample", action="store_true",
                    help="poly: time the oracle on a sample scaled by m n instead of one full-size solve")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the sub-records (PCA, batched and the method variants) of the default run")
    return apply_defaults(ap.parse_args())


def apply_defaults(a):
    dflt = {"poly": dict(prec="bf16", m=32768, n=32768, k=200, p=56, q=2, seed=2001, sample=8192),
            "pca": dict(prec="fp8b", m=1 << 20, n=4096, k=64, p=64, q=1, seed=3001, sample=32768),
            "controller": dict(prec="f32", m=0, n=0, k=0, p=0, q=0, seed=60000, sample=0),
            "batched": dict(prec="f32", m=0, n=0, k=0, p=0, q=0, seed=4001, sample=0),
            "nystrom": dict(prec="f32", m=16384, n=16384, k=200, p=56, q=0, seed=5001, sample=4096)}[a.workload]
    for key, val in dflt.items():
        if getattr(a, key) is None:
            setattr(a, key, val)
    return a


def workload_name(a):
    if a.workload == "pca":
        return ("PCA %dx%d fp32, rank-64 signal (sigma 100 -> 1) + N(0, 1e-6) noise, column-centred; "
                "k=%d p=%d (l=%d) q=%d" % (a.m, a.n, a.k, a.p, a.k + a.p, a.q))
    return "poly-decay %dx%d fp32, sigma_j=j^-1.5, Haar U,V; k=%d p=%d (l=%d) q=%d" % (
        a.m, a.n, a.k, a.p, a.k + a.p, a.q)


def make_workload(a, m, n, seed, device):
    from workloads import poly_decay_matrix, pca_matrix
    if a.workload == "pca":
        return pca_matrix(m, n, seed=seed, device=device)
    return poly_decay_matrix(m, n, seed=seed, device=device)


def sample_shape(a):
    """Shape of the CPU oracle's sample of the workload."""
    if a.workload == "pca":
        return min(a.sample, a.m), a.n
    s = min(a.sample, a.m, a.n)
    return s, s


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in a child process."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------- distributed ---
def dist_setup(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dist, device):
    """The largest x over the ranks of the process group (x itself when there
    is none): the job's time is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, units_per_rank, ms):
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units, over the slowest rank's time `ms`."""
    return world * units_per_rank / (ms / 1000.0)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------- oracle leg --
TC_PROFILE = os.path.join(ROOT, "profiles", "tc_gemm_kernel_poly_decay.md")
TC_SOURCES = [os.path.join(ROOT, "paper_1607_01649_gb300", "csrc", f) for f in ("k_tc.cu", "sm100.cuh")]


def tc_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in TC_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def tc_traffic(m, n):
    """DRAM bytes (read + write) of one sketch launch from the committed ncu
    summary, scaled from its capture size to m x n (the kernel's traffic is
    proportional to the bytes of A it streams).  None when the kernel sources
    changed since the capture or no summary exists."""
    try:
        fields = {}
        for line in open(TC_PROFILE):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        if fields.get("kernel_sources_sha256_16") != tc_source_hash():
            return None
        cm, cn = (int(x) for x in fields["capture_shape"].split("x"))
        return float(fields["dram_bytes_per_launch"]) * (m * n) / float(cm * cn)
    except Exception:
        return None


BATCH_PROFILE = os.path.join(ROOT, "profiles", "batched_kernel_kernel_blocks.md")


def profile_fields(path):
    fields = {}
    for line in open(path):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    return fields


def batched_traffic(sum_mn):
    """DRAM bytes of one batched launch from the committed ncu summary,
    scaled by the batch's sum of m n; None when the kernel source changed
    since the capture."""
    try:
        import hashlib
        f = profile_fields(BATCH_PROFILE)
        h = hashlib.sha256(open(os.path.join(ROOT, "paper_1607_01649_gb300", "csrc", "k_batched.cu"), "rb").read())
        if f.get("kernel_sources_sha256_16") != h.hexdigest()[:16]:
            return None
        return float(f["dram_bytes_per_launch"]) * sum_mn / float(f["capture_sum_mn"])
    except Exception:
        return None


def oracle_sample(a, seconds=12.0, device=None):
    """Time the float64 oracle on a sample x sample matrix of the same family
    (same k, p, q), scaled to the full workload by the m*n ratio (the sketch
    passes are linear in m*n).  Returns (solves_per_s_full_size, detail)."""
    import numpy as np
    import oracle
    sm_, sn_ = sample_shape(a)
    A = _make_matrix(a, sm_, sn_, a.seed, device).astype(np.float64) if device is not None else None
    if A is None:
        from workloads import poly_decay_matrix_np, pca_matrix_np
        A = (pca_matrix_np(sm_, sn_, a.seed) if a.workload == "pca" else
             poly_decay_matrix_np(sm_, sn_, a.seed)).astype(np.float64)
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        oracle.rsvd_power(A, a.k, a.p, a.q, a.seed)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > seconds or len(times) >= 20:
            break
    t = statistics.median(times)
    scale = (a.m * a.n) / float(sm_ * sn_)
    detail = ("float64 oracle rsvd_power on a %dx%d matrix of the same family (k=%d p=%d q=%d), %d solve(s), "
              "median %.3f s, scaled by m*n ratio %.1f" % (sm_, sn_, a.k, a.p, a.q, len(times), t, scale))
    return 1.0 / (t * scale), detail, t, len(times)


def _make_matrix(a, m, n, seed, device):
    import torch
    A = make_workload(a, m, n, seed, device)
    out = A.cpu().numpy()
    del A
    torch.cuda.empty_cache()
    return out


def run_reference(a):
    world, rank, local = dist_setup(a)
    if rank != 0:
        return
    dev = None
    try:
        import torch
        if torch.cuda.is_available():
            dev = "cuda:%d" % local
    except Exception:
        dev = None
    import numpy as np
    import oracle
    sm_, sn_ = sample_shape(a)
    if dev is not None:
        A = _make_matrix(a, sm_, sn_, a.seed, dev).astype(np.float64)
    else:
        from workloads import poly_decay_matrix_np, pca_matrix_np
        A = (pca_matrix_np(sm_, sn_, a.seed) if a.workload == "pca" else
             poly_decay_matrix_np(sm_, sn_, a.seed)).astype(np.float64)
    for _ in range(a.warmup):
        oracle.rsvd_power(A, a.k, a.p, a.q, a.seed)
    t0 = time.perf_counter()
    for i in range(a.steps):
        oracle.rsvd_power(A, a.k, a.p, a.q, a.seed + i)
    dt = time.perf_counter() - t0
    scale = (a.m * a.n) / float(sm_ * sn_)
    value = a.steps / dt / scale
    sample = ("float64 oracle rsvd_power on a %dx%d matrix of the same family (k=%d p=%d q=%d) per step, "
              "time scaled by the m*n ratio %.1f" % (sm_, sn_, a.k, a.p, a.q, scale))
    # ms_per_step is the wall time of one step as run (one sample solve); the
    # value is that rate scaled to the full-size workload by the m n ratio
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * dt / a.steps,
            "ms_per_full_size_solve": 1000.0 * dt / a.steps * scale,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def peaks():
    """HBM GB/s and bf16 TFLOP/s (burst, sustained): MEASURED_PEAKS.json, else
    the profiling recipe's fallback figures."""
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return (float(pk["hbm_gbs"]), float(pk["bf16_tflops"]), float(pk.get("bf16_tflops_sustained", pk["bf16_tflops"])),
                "measured")
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def solve_roofline(m, n, l, q, passes, bytes_per_entry, ms_per_step, fp8=False):
    """The per-solve floor of the method: the slower of its sketch flops at the
    tensor-core peak (sustained: the solve is timed inside a long loop; e4m3
    at twice the bf16 rate) and its passes over A at the HBM copy bandwidth,
    divided by the measured time per solve; beside it the compulsory floor
    (A read once in its given fp32 form)."""
    hbm, _, tc_s, src = peaks()
    tc = tc_s * (2.0 if fp8 else 1.0)
    flops = passes * 2.0 * m * n * l
    t_flop = flops / (tc * 1e12) * 1e3
    t_bytes = passes * bytes_per_entry * m * n / (hbm * 1e9) * 1e3
    floor = max(t_flop, t_bytes)
    t_comp = 4.0 * m * n / (hbm * 1e9) * 1e3
    return {"floor_ms": floor, "frac": floor / ms_per_step, "bound": "hbm" if t_bytes >= t_flop else "tensor",
            "passes_over_A": passes, "bytes_per_entry": bytes_per_entry, "sketch_flops": flops,
            "compulsory_floor_ms": t_comp, "compulsory_frac": t_comp / ms_per_step, "peak_source": src}


# ------------------------------------------------------------------- ours --
def run_ours(a):
    import numpy as np
    import torch
    import paper_1607_01649_gb300 as rs

    world, rank, local = dist_setup(a)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    else:
        dist = None

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    m, n, k, p, q = a.m, a.n, a.k, a.p, a.q
    l = k + p
    prec = {"bf16": rs.RSVD_MIXED_BF16, "fp8": rs.RSVD_MIXED_FP8, "fp8b": rs.RSVD_MIXED_FP8_B128,
            "f32": rs.RSVD_F32}[a.prec]
    fp8 = prec in (rs.RSVD_MIXED_FP8, rs.RSVD_MIXED_FP8_B128)
    A = make_workload(a, m, n, a.seed + rank, dev)
    h = rs.handle(local)
    prm = rs.make_params(k, p, q, seed=a.seed, prec=prec, flags=0)
    ws = torch.empty(rs.rsvd_workspace_size(h, m, n, prm), dtype=torch.uint8, device=dev)
    U = torch.empty(m, k, dtype=torch.float32, device=dev)
    D = torch.empty(k, dtype=torch.float64, device=dev)
    V = torch.empty(n, k, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def solve(seed):
        prm.seed = seed
        code = rs.rsvd_fixed_rank(h, m, n, A, A.stride(0), prm, U, U.stride(0), D, V, V.stride(0), ws)
        if code != rs.RSVD_OK:
            raise rs.RsvdError(code, rs.last_error(h))

    for i in range(a.warmup):
        solve(a.seed + i)
    torch.cuda.synchronize()
    st = rs.rsvd_query_status(h, ws)
    if st != rs.RSVD_OK:
        raise rs.RsvdError(st, "device status after warm-up")

    # ---- timed region
    clocks = ClockSampler(torch.cuda.current_device())
    rs.rsvd_profile_read(h, 0)
    rs.rsvd_profile_read(h, 1)
    rs.rsvd_profile(h, 1)
    launches0 = rs.rsvd_kernel_launches(h)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(a.steps):
        solve(a.seed + 100 + i)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    rs.rsvd_profile(h, 0)
    launches = rs.rsvd_kernel_launches(h) - launches0
    ms = e0.elapsed_time(e1)
    sk_ms, sk_n = rs.rsvd_profile_read(h, 0)
    pj_ms, pj_n = rs.rsvd_profile_read(h, 1)
    ms = max_over_ranks(ms, dist, dev)
    st = rs.rsvd_query_status(h, ws)
    if st != rs.RSVD_OK:
        raise rs.RsvdError(st, "device status after timing")
    ms_per_step = ms / a.steps
    value = replica_throughput(world, a.steps, ms)
    diag = rs.status_block(ws)

    # ---- accuracy of the last solve (not timed): singular values against the
    # construction, Frobenius residual in float64 blockwise
    torch.cuda.synchronize()

    def fro_rel(Uo, Do, Vo):
        f2, a2 = 0.0, 0.0
        Ud = (Uo.double() * Do[None, :])
        for r0 in range(0, m, 4096):
            Ab = A[r0:r0 + 4096].double()
            R = Ab - Ud[r0:r0 + 4096] @ Vo.double().T
            f2 += float((R * R).sum())
            a2 += float((Ab * Ab).sum())
        return (f2 / a2) ** 0.5, a2 ** 0.5

    def spectral_rel(Uo, Do, Vo, iters=30, b=4):
        """||A - U D V^T||_2 / ||A||_2 by a randomized block power iteration
        (b columns, `iters` steps) with the factorization applied implicitly:
        products with A in binary32 (no TF32; A is binary32 data), everything
        else in float64.  Returns (estimate, last relative change of the
        estimate, ||A||_2 estimate)."""
        g = torch.Generator(device=dev)
        g.manual_seed(12345)
        Ud, Vd, Dd = Uo.double(), Vo.double(), Do.double()
        prev_tf32 = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False

        def apply(X, resid, trans):
            out = (A.T @ X.float() if trans else A @ X.float()).double()
            if resid:
                out -= (Vd @ (Dd[:, None] * (Ud.T @ X))) if trans else (Ud @ (Dd[:, None] * (Vd.T @ X)))
            return out

        def power(resid):
            X = torch.randn(n, b, dtype=torch.float64, device=dev, generator=g)
            est, prev = 0.0, 0.0
            for _ in range(iters):
                X, _ = torch.linalg.qr(X)
                Y = apply(X, resid, False)
                Z = apply(Y, resid, True)
                prev, est = est, float(torch.linalg.norm(Z, 2, dim=0).max()) ** 0.5
                X = Z
            return est, abs(est - prev) / est if est > 0 else 0.0

        try:
            r, conv = power(True)
            a2, _ = power(False)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev_tf32
        return r / a2, conv, a2

    res_rel, fro_a = fro_rel(U, D, V)
    spec_rel, spec_conv, spec_a = spectral_rel(U, D, V)

    def orth_err(X):
        # max |X^T X - I| in float64
        X64 = X.double()
        return float((X64.T @ X64 - torch.eye(X64.shape[1], dtype=torch.float64, device=dev)).abs().max())

    orth = {"max_abs(U^T U - I)": orth_err(U), "max_abs(V^T V - I)": orth_err(V)}
    if a.workload == "pca":
        # the signal's singular values (the noise moves them by about its norm)
        sig_true = torch.linspace(100.0, 1.0, 64, dtype=torch.float64, device=dev)[:k]
        nk = min(k, 48)
        d_rel = float(((D[:nk] - sig_true[:nk]).abs() / sig_true[:nk]).max())
        err = {"max_rel_err_sigma_1..48_vs_signal": d_rel, "fro_residual_rel": res_rel,
               "noise_floor_rel": 1e-3 * (m * n) ** 0.5 / fro_a,
               "spectral_residual_rel": spec_rel, "spectral_estimate_last_rel_change": spec_conv,
               "sigma_k+1_rel(noise, sqrt(m)+sqrt(n) times 1e-3)": 1e-3 * (m ** 0.5 + n ** 0.5) / spec_a, **orth}
    else:
        sig_true = torch.arange(1, k + 1, dtype=torch.float64, device=dev).pow(-1.5)
        d_rel = float(((D - sig_true).abs() / sig_true).max())
        fro_opt = float(torch.arange(k + 1, min(m, n) + 1, dtype=torch.float64).pow(-3.0).sum().sqrt())
        err = {"max_rel_err_sigma_1..k_vs_construction": d_rel, "fro_residual_rel": res_rel,
               "fro_residual_optimal_rel(Eckart-Young)": fro_opt / fro_a,
               "spectral_residual_rel": spec_rel, "spectral_estimate_last_rel_change": spec_conv,
               "sigma_k+1_rel(Eckart-Young)": (k + 1) ** -1.5, **orth}

    # ---- roofline of the dominant kernel: the tcgen05 sketch product
    roof = None
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
        peak_src = "measured"
    except Exception:
        hbm, peak_src = 6800.0, "fallback"
    if (prec == rs.RSVD_MIXED_BF16 or fp8) and sk_n > 0:
        per_launch_ms = sk_ms / sk_n
        # algorithmic bytes of the sketch products of one solve: A once per
        # product (bf16: 2 bytes, e4m3: 1 byte per entry), the thin operand in the
        # same type, the fp32 output; q + 1 products A X (m x l out), q products
        # A^T X (n x l out); averaged per launch
        eb = 2.0 if prec == rs.RSVD_MIXED_BF16 else 1.0
        nn_b = eb * m * n + eb * n * l + 4.0 * m * l
        tn_b = eb * m * n + eb * m * l + 4.0 * n * l
        alg_bytes = ((q + 1) * nn_b + q * tn_b) / (2 * q + 1)
        achieved = alg_bytes / (per_launch_ms / 1000.0) / 1e9
        kname = ("tc_gemm_kernel (bf16 sketch A*X / A^T*X, stream-K)" if prec == rs.RSVD_MIXED_BF16 else
                 "tc_gemm_kernel<..., F8> (e4m3 sketch A8*X8t^T, kind::f8f6f4, stream-K)")
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": tc_traffic(m, n) if prec == rs.RSVD_MIXED_BF16 else None,
                "algorithmic_bytes": alg_bytes, "kernel": kname,
                "launches": sk_n, "avg_ms": per_launch_ms, "peak_source": peak_src,
                "projection_split3_avg_ms": (pj_ms / pj_n) if pj_n else None}
        # the whole solve against the method's floor: 2q + 2 passes over A
        # (q + 1 products A X, q products A^T X, the projection) at the
        # sketch's bytes per entry
        sr = solve_roofline(m, n, l, q, 2 * q + 2, eb, ms_per_step, fp8=fp8)
        roof["solve_frac"] = sr["frac"]
        roof["solve"] = sr
        # and against this design's own bytes: the conversion pass (fp32 A read,
        # the bf16 pair written; e4m3 also writes A8 and its byte transpose),
        # the 2q + 1 sketch passes and the split-bf16 projection (Ah + Al)
        conv = (8.0 if prec == rs.RSVD_MIXED_BF16 else 11.0) * m * n
        if prec == rs.RSVD_MIXED_FP8_B128:
            conv += 4.0 * m * n  # the read of A that finds the 128-row block maxima
        design_bytes = conv + (2 * q + 1) * eb * m * n + 4.0 * m * n
        roof["solve_design_floor_ms"] = design_bytes / (hbm * 1e9) * 1e3
        roof["solve_design_frac"] = roof["solve_design_floor_ms"] / ms_per_step
    elif prec == rs.RSVD_F32:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "traffic": None}

    variants = None
    if not a.no_extra and world == 1:
        if a.workload == "poly":
            variants = poly_variants(a, rs, h, A, dev, stream, fro_rel)
        elif a.workload == "pca":
            variants = {"centring": pca_centring(a, rs, h, A, dev, stream, D)}
            if prec == rs.RSVD_MIXED_FP8_B128:
                variants["e4m3_per_row_scales"] = pca_per_row(a, rs, h, A, dev, stream, D)

    # ---- e2e: the C-ABI call with HOST buffers (pinned).  The mixed paths read
    # A exactly once, in the conversion pass, so A is passed as the host
    # pointer and read over the host link inside that pass (no device copy);
    # U, D, V are written to host memory by the kernels.  The binary32 path
    # reads A 2q + 2 times, so there A is copied in and U, D, V copied out.
    e2e = None
    if not a.no_e2e:
        Ah = torch.empty(m, n, dtype=torch.float32, pin_memory=True)
        Ah.copy_(A)
        Uh = torch.empty(m, k, dtype=torch.float32, pin_memory=True)
        Dh = torch.empty(k, dtype=torch.float64, pin_memory=True)
        Vh = torch.empty(n, k, dtype=torch.float32, pin_memory=True)
        zero_copy = prec == rs.RSVD_MIXED_BF16 or fp8
        steps_e2e = max(1, min(a.steps, 5))
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(steps_e2e):
            if zero_copy:
                prm.seed = a.seed + 200 + i
                code = rs.rsvd_fixed_rank(h, m, n, Ah, n, prm, Uh, k, Dh, Vh, k, ws)
                if code != rs.RSVD_OK:
                    raise rs.RsvdError(code, rs.last_error(h))
            else:
                A.copy_(Ah, non_blocking=True)
                solve(a.seed + 200 + i)
                Uh.copy_(U, non_blocking=True)
                Dh.copy_(D, non_blocking=True)
                Vh.copy_(V, non_blocking=True)
        f1.record(stream)
        barrier()
        ems = max_over_ranks(f0.elapsed_time(f1), dist, dev)
        e2e = {"value": replica_throughput(world, steps_e2e, ems), "unit": "solves/s",
               "h2d_bytes_per_step": m * n * 4, "d2h_bytes_per_step": (m * k + n * k) * 4 + k * 8,
               "steps": steps_e2e,
               "mode": ("pinned host A, U, D, V passed to rsvd_fixed_rank; A read over the host link by the "
                        "conversion pass" if zero_copy else "pinned host A copied in, U, D, V copied out")}
        del Ah

    # ---- comparators on the same matrix (1 timed solve each): the plain
    # binary32 SIMT path, and for the e4m3 workload also the bf16 path
    def comparator(pc):
        prm2 = rs.make_params(k, p, q, seed=a.seed, prec=pc, flags=0)
        ws2 = torch.empty(rs.rsvd_workspace_size(h, m, n, prm2), dtype=torch.uint8, device=dev)
        U2, D2, V2 = torch.empty_like(U), torch.empty_like(D), torch.empty_like(V)
        rs.rsvd_fixed_rank(h, m, n, A, A.stride(0), prm2, U2, k, D2, V2, k, ws2)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        rs.rsvd_fixed_rank(h, m, n, A, A.stride(0), prm2, U2, k, D2, V2, k, ws2)
        g1.record(stream)
        torch.cuda.synchronize()
        nk = min(k, 48) if a.workload == "pca" else k
        d2 = float(((D2[:nk] - sig_true[:nk]).abs() / sig_true[:nk]).max())
        out = {"value": 1000.0 / g0.elapsed_time(g1), "unit": "solves/s", "max_rel_err_sigma": d2,
               "fro_residual_rel": fro_rel(U2, D2, V2)[0]}
        del ws2
        return out

    f32 = comparator(rs.RSVD_F32) if (prec != rs.RSVD_F32 and not a.no_f32) else None
    bf16 = comparator(rs.RSVD_MIXED_BF16) if (fp8 and not a.no_f32) else None

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    cpu = None
    if not a.no_cpu:
        if a.workload == "poly" and not a.cpu_sample:
            cpu = oracle_full(a, A, a.seed + 100 + a.steps - 1, D, res_rel, fro_rel, dev)
        else:
            v, detail, t, nsol = oracle_sample(a, device=dev)
            cpu = {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle", "sample": detail}
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e4m3" if fp8 else ("bf16" if prec == rs.RSVD_MIXED_BF16 else "f32"),
            "data": "synthetic",
            "config": {"workload": workload_name(a), "precision": a.prec,
                       "l2": "inputs larger than L2 (A is %.2f GB; L2 129 MB)" % (m * n * 4 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "error": err, "plain_f32": f32, "mixed_bf16": bf16,
            "diagnostics": {"jacobi_sweeps_last_solve": diag["jacobi_sweeps"],
                            "shifted_cholesky_last_solve": diag["shift_count"],
                            "sketch_launches_timed": sk_n, "projection_launches_timed": pj_n}}
    if variants is not None:
        line["variants"] = variants
    if dist is not None:
        dist.destroy_process_group()
    return line


def oracle_full(a, A, seed, D_gpu, res_gpu, fro_rel, dev):
    """One full-size float64 oracle solve (oracle.rsvd_power, Fig.
    RSVDP_stabilized) on the host cores, on the same binary32 A (promoted to
    float64) and the same Omega seed as the last timed GPU solve; its own
    error beside the GPU's."""
    import numpy as np
    import torch
    import oracle
    A64 = A.double().cpu().numpy()
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    ref = oracle.rsvd_power(A64, a.k, a.p, a.q, seed)
    t = time.perf_counter() - t0
    del A64
    Ur = torch.from_numpy(ref["U"]).to(dev)
    Vr = torch.from_numpy(ref["V"]).to(dev)
    Dr = torch.from_numpy(ref["D"]).to(dev)
    res_ref, _ = fro_rel(Ur, Dr, Vr)
    sig = torch.arange(1, a.k + 1, dtype=torch.float64, device=dev).pow(-1.5)
    d_ref = float(((Dr - sig).abs() / sig).max())
    gpu_vs = float(((D_gpu.double() - Dr).abs() / Dr).max())
    return {"value": 1.0 / t, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": "one full-size float64 oracle solve (rsvd_power, %dx%d, k=%d p=%d q=%d) on the same A and "
                      "Omega seed as the last timed GPU solve: %.1f s" % (a.m, a.n, a.k, a.p, a.q, t),
            "oracle_error": {"fro_residual_rel": res_ref, "max_rel_err_sigma_1..k_vs_construction": d_ref},
            "gpu_error_vs_oracle": {"fro_residual_ratio": res_gpu / res_ref, "max_rel_diff_sigma_1..k": gpu_vs}}


def _timed(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def poly_variants(a, rs, h, A, dev, stream, fro_rel):
    """The method variants of the paper on the same poly-decay matrix (bf16
    tensor-core sketches, one rsvd_fixed_rank call per solve, 5 timed), each
    with its passes over A, its solve roofline fraction and its Frobenius
    residual against the Eckart-Young optimum at its rank k:
    * power_q1_l256 / power_q2_l256: Fig. RSVDP_stabilized, k = 120;
    * krylov_2x128: the extended sampling matrix, 2 blocks of 128 columns
      (the same 4 passes as q = 1 at width 256);
    * basic_q0_l128: Fig. RSVD, k = 120, p = 8 (2 passes);
    * single_pass_l256: Fig. singlepass_gen, k = 120, p = 136 (the two
      sketches as separate launches: 2 reads of A; with p = 8 the fit of
      the core from bf16 sketches is too poorly conditioned to be useful);
    * srft_l128: Fig. RSVD with the SRFT test matrix, k = 100, p = 28
      (complex factors);
    * adaptive_spectral_4096: rsvd_adaptive_tol in its spectral mode on a
      4096^2 exp(-j/20)-decay matrix (binary32; a j^-1.5 tail keeps the
      Frobenius norm of the remainder, which the probes see, far above a
      spectral eps at any rank under 256), eps = 5e-3 ||A||_2."""
    import torch
    m, n = a.m, a.n
    out = {}
    fro_a2 = float(torch.arange(1, min(m, n) + 1, dtype=torch.float64).pow(-3.0).sum())

    def opt_rel(k):
        return float(torch.arange(k + 1, min(m, n) + 1, dtype=torch.float64).pow(-3.0).sum().sqrt()) / fro_a2 ** 0.5

    cases = [("power_q1_l256", dict(k=120, p=136, q=1), 4, 256),
             ("power_q2_l256", dict(k=120, p=136, q=2), 6, 256),
             ("krylov_2x128", dict(k=120, p=8, q=2, krylov=True), 4, 256),
             ("basic_q0_l128", dict(k=120, p=8, q=0), 2, 128),
             ("single_pass_l256", dict(k=120, p=136, q=0, single_pass=True), 2, 256),
             ("srft_l128", dict(k=100, p=28, q=0, srft=True), 2, 256)]
    for name, kw, passes, width in cases:
        try:
            kw = dict(kw)
            k = kw.pop("k")
            p_ = kw.pop("p")
            q_ = kw.pop("q")
            flags = ((rs.RSVD_FLAG_KRYLOV if kw.get("krylov") else 0) |
                     (rs.RSVD_FLAG_SINGLE_PASS if kw.get("single_pass") else 0) |
                     (rs.RSVD_FLAG_SRFT if kw.get("srft") else 0))
            prm = rs.make_params(k, p_, q_, seed=a.seed, prec=rs.RSVD_MIXED_BF16, flags=flags)
            ws = torch.empty(rs.rsvd_workspace_size(h, m, n, prm), dtype=torch.uint8, device=dev)
            dt = torch.complex64 if kw.get("srft") else torch.float32
            U = torch.empty(m, k, dtype=dt, device=dev)
            D = torch.empty(k, dtype=torch.float64, device=dev)
            V = torch.empty(n, k, dtype=dt, device=dev)

            def solve():
                code = rs.rsvd_fixed_rank(h, m, n, A, A.stride(0), prm, U, k, D, V, k, ws)
                if code != rs.RSVD_OK:
                    raise rs.RsvdError(code, rs.last_error(h))

            ms = _timed(solve, 5, stream)
            if kw.get("srft"):
                f2, a2 = 0.0, 0.0
                Ud = U.to(torch.complex128) * D[None, :]
                for r0 in range(0, m, 4096):
                    Ab = A[r0:r0 + 4096].double()
                    R = Ab - (Ud[r0:r0 + 4096] @ V.to(torch.complex128).conj().T).real
                    f2 += float((R * R).sum())
                    a2 += float((Ab * Ab).sum())
                res = (f2 / a2) ** 0.5
            else:
                res = fro_rel(U, D, V)[0]
            sr = solve_roofline(m, n, width, 0, passes, 2.0, ms)
            out[name] = {"value": 1000.0 / ms, "unit": "solves/s", "ms": ms, "k": k, "basis_width": width,
                         "passes_over_A": passes, "solve_frac": sr["frac"], "fro_residual_rel": res,
                         "fro_optimal_rel": opt_rel(k), "ratio_to_optimal": res / opt_rel(k)}
            del ws, U, D, V
            torch.cuda.empty_cache()
        except Exception as exc:  # a variant that fails is reported, not fatal
            out[name] = {"error": str(exc)[:200]}
    try:
        from workloads import exp_decay_matrix_torch
        As = exp_decay_matrix_torch(4096, 4096, seed=a.seed + 7, rate=20.0, device=dev)
        # 5e-3 sigma_1: the probe test (max of 16 fresh probes at most
        # eps / (10 sqrt(2/pi))) then stops at rank 208; at 1e-3 sigma_1 the
        # blocked finder needs more than 256 columns on this spectrum (the
        # float64 oracle's probes, same seeds: 1.25e-4 at rank 240 against a
        # threshold of 1.19e-4)
        eps = 5e-3 * float(torch.exp(torch.tensor(-1.0 / 20.0)))
        res = {}

        def solve_spec():
            res["r"] = rs.adaptive_tol(As, eps, block=16, seed=a.seed, prec=rs.RSVD_F32, spectral=True)

        ms = _timed(solve_spec, 3, stream)
        U, D, V, rank, bound, code = res["r"]
        Ud = U[:, :rank].double() * D[:rank][None, :]
        E = As.double() - Ud @ V[:, :rank].double().T
        true2 = float(torch.linalg.matrix_norm(E, 2))
        out["adaptive_spectral_4096"] = {"value": 1000.0 / ms, "unit": "solves/s", "ms": ms, "eps": eps,
                                         "rank": rank, "status": code, "reported_bound": bound,
                                         "true_spectral_error": true2,
                                         "sigma_rank+1": float(torch.exp(torch.tensor(-(rank + 1) / 20.0)))}
        del As, E
        torch.cuda.empty_cache()
    except Exception as exc:
        out["adaptive_spectral_4096"] = {"error": str(exc)[:200]}
    return out


def pca_per_row(a, rs, h, A, dev, stream, D_block):
    """The same PCA solve with one e4m3 scale per row of A instead of per
    128-row block (one read of A fewer): time and the singular values beside
    the block-scaled solve's."""
    import torch
    m, n, k, p, q = a.m, a.n, a.k, a.p, a.q
    prm = rs.make_params(k, p, q, seed=a.seed + 100 + a.steps - 1, prec=rs.RSVD_MIXED_FP8, flags=0)
    ws = torch.empty(rs.rsvd_workspace_size(h, m, n, prm), dtype=torch.uint8, device=dev)
    U = torch.empty(m, k, dtype=torch.float32, device=dev)
    D = torch.empty(k, dtype=torch.float64, device=dev)
    V = torch.empty(n, k, dtype=torch.float32, device=dev)

    def solve():
        code = rs.rsvd_fixed_rank(h, m, n, A, A.stride(0), prm, U, k, D, V, k, ws)
        if code != rs.RSVD_OK:
            raise rs.RsvdError(code, rs.last_error(h))

    ms = _timed(solve, 5, stream)
    nk = min(k, 48)
    diff = float(((D[:nk] - D_block[:nk]).abs() / D_block[:nk]).max())
    del ws, U, V
    return {"value": 1000.0 / ms, "unit": "solves/s", "ms": ms,
            "max_rel_diff_sigma_1..48_vs_block_scaled": diff}


def pca_centring(a, rs, h, A, dev, stream, D_centred):
    """PCA as it arrives: the same matrix with column offsets added (entry
    scale), factored with implicit centring (RSVD_FLAG_CENTER) in the
    benchmark's precision; its singular values against those of the solve on
    the explicitly centred matrix, and the time beside it."""
    import torch
    from workloads import column_offsets
    m, n, k, p, q = a.m, a.n, a.k, a.p, a.q
    prec = {"bf16": rs.RSVD_MIXED_BF16, "fp8": rs.RSVD_MIXED_FP8, "fp8b": rs.RSVD_MIXED_FP8_B128,
            "f32": rs.RSVD_F32}[a.prec]
    fp8 = prec in (rs.RSVD_MIXED_FP8, rs.RSVD_MIXED_FP8_B128)
    scale = float(A[:4096].double().pow(2).mean().sqrt())
    mu = column_offsets(n, a.seed + 11, 2.0 * scale, device=dev)
    A.add_(mu[None, :])
    try:
        prm = rs.make_params(k, p, q, seed=a.seed + 100 + a.steps - 1, prec=prec, flags=rs.RSVD_FLAG_CENTER)
        ws = torch.empty(rs.rsvd_workspace_size(h, m, n, prm), dtype=torch.uint8, device=dev)
        U = torch.empty(m, k, dtype=torch.float32, device=dev)
        D = torch.empty(k, dtype=torch.float64, device=dev)
        V = torch.empty(n, k, dtype=torch.float32, device=dev)

        def solve():
            code = rs.rsvd_fixed_rank(h, m, n, A, A.stride(0), prm, U, k, D, V, k, ws)
            if code != rs.RSVD_OK:
                raise rs.RsvdError(code, rs.last_error(h))

        ms = _timed(solve, 5, stream)
        nk = min(k, 48)
        diff = float(((D[:nk] - D_centred[:nk]).abs() / D_centred[:nk]).max())
        one_u = float(U.double().sum(dim=0).abs().max() / m ** 0.5)
        del ws, U, V
        return {"value": 1000.0 / ms, "unit": "solves/s", "ms": ms, "offset_scale": 2.0 * scale,
                "max_rel_diff_sigma_1..48_vs_explicitly_centred": diff, "max_abs_1^T_u_over_sqrt_m": one_u}
    finally:
        A.sub_(mu[None, :])


# ------------------------------------------------------- controller stream --
def run_controller(a):
    """Trains the controller on the GPU from the adaptive finder's own labels
    (training seeds 50000+), then solves a held-out stream (seeds a.seed +
    i, `steps` matrices, n log-uniform in [lo, hi]) to relative Frobenius
    tolerance 1e-4 four ways: the controller (probe, network, fixed-rank
    solve, judge, and the adaptive range finder as fallback), the same with
    the escalating fallback (one more fixed-rank solve at l = 256, q >= 2),
    the blocked adaptive range finder alone, and a fixed conservative
    l = min(n, 256), q = 2.  Matrices are synthesized
    before each solve (untimed); solves are timed with CUDA events."""
    import numpy as np
    import torch
    import paper_1607_01649_gb300 as rs
    from workloads import controller_matrix, mlp_init
    dev = torch.device("cuda", 0)
    h = rs.handle(0)
    tol = 1e-4
    X, yl, yq = [], [], []
    t0 = time.perf_counter()
    for s in range(50000, 50000 + a.train):
        A, _ = controller_matrix(s, lo=a.lo, hi=a.hi, device=dev)
        f, _ = rs.probe_features(A, seed=s)
        X.append(f)
        _, _, (c, q) = rs.adaptive_labels(A, tol, seed=s, max_rank=min(A.shape[0], 256))
        yl.append(c)
        yq.append(q)
        del A
    X = torch.stack(X)
    yl = torch.tensor(yl, dtype=torch.int32, device=dev)
    yq = torch.tensor(yq, dtype=torch.int32, device=dev)
    theta = torch.from_numpy(mlp_init(7).astype(np.float32)).to(dev)
    tr = rs.Trainer(theta, lr=2e-3, lam=1.0)
    for _ in range(3000):
        tr.step(X, yl, yq)
    loss = float(tr.step(X, yl, yq).item())
    t_train = time.perf_counter() - t0

    def rel_residual(A, U, D, V, r):
        f2, a2 = 0.0, 0.0
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            UD = U[:, :r] * D[:r].float()[None, :]
            for r0 in range(0, A.shape[0], 4096):
                Ab = A[r0:r0 + 4096]
                R = Ab - UD[r0:r0 + 4096] @ V[:, :r].T
                f2 += float((R.double() ** 2).sum())
                a2 += float((Ab.double() ** 2).sum())
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
        return (f2 / a2) ** 0.5

    stream = torch.cuda.current_stream()
    res = {"adaptive": [0.0, 0, 0], "controller": [0.0, 0, 0], "escalate": [0.0, 0, 0], "fixed": [0.0, 0, 0]}
    falls = {"controller": 0, "escalate": 0}
    for i in range(a.warmup + a.steps):
        s = a.seed + i
        A, _ = controller_matrix(s, lo=a.lo, hi=a.hi, device=dev)
        n = A.shape[0]
        R = min(n, 256)
        for meth in ("adaptive", "controller", "escalate", "fixed"):
            rs.rsvd_controller_attach(h, tr.theta, 0.9, 0.8)
            rs.rsvd_controller_fallback(h, 1 if meth == "escalate" else 0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if meth == "adaptive":
                U, D, V, r, err, code = rs.adaptive_tol(A, tol, seed=s, max_rank=R)
            elif meth in ("controller", "escalate"):
                U, D, V, r, err, code = rs.adaptive_tol(A, tol, seed=s, max_rank=R, controller=True)
            else:
                U, D, V = rs.fixed_rank(A, R, 0, 2, seed=s, full=True, sync=True)
                r = R
            e1.record(stream)
            torch.cuda.synchronize()
            if i < a.warmup:
                continue
            if meth in ("controller", "escalate"):
                info = rs.rsvd_controller_last(h)
                falls[meth] += info["fallback"] or info["escalated"]
            res[meth][0] += e0.elapsed_time(e1)
            res[meth][1] += 1
            res[meth][2] += rel_residual(A, U, D, V, r) <= tol
            del U, D, V
        del A
    out = {m: {"solves_per_s": v[1] / (v[0] / 1000.0), "fraction_meeting_tol": v[2] / max(v[1], 1)}
           for m, v in res.items()}
    line = {"metric": METRIC, "value": out["controller"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": res["controller"][0] / max(res["controller"][1], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": controller_name(a, a.steps),
                       "training": "%d matrices, labels from the adaptive finder (q = 0..3), 3000 Adam steps, "
                                   "final loss %.3f, %.0f s" % (a.train, loss, t_train)},
            "controller": out["controller"], "controller_escalating": out["escalate"],
            "adaptive_only": out["adaptive"], "fixed_l256_q2": out["fixed"], "fallbacks": falls,
            "cpu_baseline": None if a.no_cpu else controller_cpu_baseline(a, 20.0)}
    print(json.dumps(line))


CONTROLLER_TOL = 1e-4
CONTROLLER_CAP = 1024


def controller_oracle_solve(a, i):
    """Matrix i of the held-out stream (seed a.seed + i: its size n and its
    spectrum) solved to the stream's tolerance by the float64 oracle's blocked
    adaptive range finder -- the method without the learned part -- on an
    n' x n' stand-in, n' = min(n, 1024), with the spectrum's first n' values
    and Haar factors.  Returns (time scaled to n x n by (n / n')^2, n)."""
    import oracle
    from workloads import controller_case, lowrank_np
    s = a.seed + i
    n, sig, _, _ = controller_case(s, a.lo, a.hi)
    ns = min(n, CONTROLLER_CAP)
    A = lowrank_np(ns, ns, sig[:ns], s)
    t0 = time.perf_counter()
    oracle.adaptive_blocked(A, CONTROLLER_TOL, b=16, seed=s, max_rank=min(ns, 256))
    return (time.perf_counter() - t0) * (n / float(ns)) ** 2, n


def controller_sample_text(count, mean_n):
    return ("float64 oracle adaptive_blocked (b=16, tol %.0e, max rank 256) on the first %d timed matrices of the "
            "held-out stream (mean n %.0f), each on a stand-in with n capped at %d (same spectrum, Haar factors), "
            "time scaled by (n / n')^2" % (CONTROLLER_TOL, count, mean_n, CONTROLLER_CAP))


def controller_name(a, steps):
    return ("controller stream: %d held-out square fp32 matrices, n log-uniform in [%d, %d], spectra exp / poly / "
            "step, tol 1e-4 relative Frobenius" % (steps, a.lo, a.hi))


def controller_cpu_baseline(a, seconds):
    """The oracle timed on the stream's timed matrices (a.warmup, a.warmup +
    1, ...), one after another, for about `seconds`; returns the cpu_baseline
    dict."""
    t0 = time.perf_counter()
    scaled, ns = 0.0, []
    while time.perf_counter() - t0 < seconds and len(ns) < a.steps:
        t, n = controller_oracle_solve(a, a.warmup + len(ns))
        scaled += t
        ns.append(n)
    return {"value": len(ns) / scaled, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": controller_sample_text(len(ns), sum(ns) / float(len(ns)))}


def run_reference_controller(a):
    """The oracle arm for the controller stream: the same matrices as the
    GPU arm, warm-up steps on the first a.warmup, step i on a.warmup + i."""
    world, rank, local = dist_setup(a)
    if rank != 0:
        return
    for w in range(a.warmup):
        controller_oracle_solve(a, w)
    scaled, ns = 0.0, []
    for i in range(a.steps):
        t, n = controller_oracle_solve(a, a.warmup + i)
        scaled += t
        ns.append(n)
    value = a.steps / scaled
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * scaled / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": controller_name(a, a.steps)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": controller_sample_text(a.steps, sum(ns) / float(a.steps))},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------- nystrom -------
def nystrom_oracle_solve(a, As, seed):
    """One float64 oracle Nystrom solve on the ns x ns sample As; returns its
    time scaled to the n x n workload by the n^2 ratio."""
    import oracle
    t0 = time.perf_counter()
    oracle.nystrom(As, a.k, a.p, seed)
    return (time.perf_counter() - t0) * (a.n / float(As.shape[0])) ** 2


def nystrom_sample_text(a, ns, reps, scaled_s):
    return ("float64 oracle nystrom on a %dx%d SPD matrix of the same family (k=%d p=%d), %d solve(s), %.3f s "
            "each, scaled by the n^2 ratio %.1f" % (ns, ns, a.k, a.p, reps,
                                                    scaled_s / (a.n / float(ns)) ** 2, (a.n / float(ns)) ** 2))


def run_reference_nystrom(a):
    """The oracle arm for the Nystrom workload: each step is one float64
    oracle solve on an a.sample x a.sample matrix of the same SPD family,
    timed on the host cores and scaled by the n^2 ratio."""
    world, rank, local = dist_setup(a)
    if rank != 0:
        return
    from workloads import spd_matrix_np
    ns = min(a.sample, a.n)
    As = spd_matrix_np(ns, seed=a.seed)
    for i in range(a.warmup):
        nystrom_oracle_solve(a, As, a.seed + i)
    scaled = sum(nystrom_oracle_solve(a, As, a.seed + 100 + i) for i in range(a.steps))
    value = a.steps / scaled
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * scaled / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": nystrom_name(a)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": nystrom_sample_text(a, ns, a.steps, scaled / a.steps)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def nystrom_name(a):
    return ("Nystrom EVD (Fig. nystrom), SPD %dx%d fp32 = V diag(j^-1.5) V^T, Haar V; k=%d p=%d (l=%d)"
            % (a.n, a.n, a.k, a.p, a.k + a.p))


def run_nystrom(a):
    """rsvd_nystrom (Fig. nystrom) on a 16384^2 SPD matrix V diag(j^-1.5) V^T,
    binary32; beside it the fixed-rank RSVD with the same two passes over A
    (q = 0) and with one power step (q = 1), their spectral residuals, and the
    float64 oracle on a sample."""
    import numpy as np
    import torch
    import paper_1607_01649_gb300 as rs
    from workloads import spd_matrix, spd_matrix_np
    dev = torch.device("cuda", 0)
    n, k, p = a.n, a.k, a.p
    l = k + p
    A = spd_matrix(n, seed=a.seed, device=dev)
    h = rs.handle(0)
    prm = rs.make_params(k, p, 0, seed=a.seed, prec=rs.RSVD_F32, flags=0)
    ws = torch.empty(rs.rsvd_workspace_size(h, n, n, prm), dtype=torch.uint8, device=dev)
    U = torch.empty(n, k, device=dev)
    L = torch.empty(k, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def solve(seed):
        prm.seed = seed
        code = rs.rsvd_nystrom(h, n, A, n, prm, U, k, L, ws)
        if code != rs.RSVD_OK:
            raise rs.RsvdError(code, rs.last_error(h))

    for i in range(a.warmup):
        solve(a.seed + i)
    torch.cuda.synchronize()
    launches0 = rs.rsvd_kernel_launches(h)
    clocks = ClockSampler(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(a.steps):
        solve(a.seed + 100 + i)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = rs.rsvd_kernel_launches(h) - launches0
    st = rs.rsvd_query_status(h, ws)
    if st != rs.RSVD_OK:
        raise rs.RsvdError(st, "device status after timing")

    def spectral(apply_resid, iters=30, b=4):
        g = torch.Generator(device=dev)
        g.manual_seed(7)
        X = torch.randn(n, b, dtype=torch.float64, device=dev, generator=g)
        est = prev = 0.0
        for _ in range(iters):
            X, _ = torch.linalg.qr(X)
            Z = apply_resid(apply_resid(X))
            prev, est = est, float(torch.linalg.norm(Z, 2, dim=0).max()) ** 0.5
            X = Z
        return est, abs(est - prev) / est if est > 0 else 0.0

    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        Ud, Ld = U.double(), L.double()
        ny, ny_conv = spectral(lambda X: (A @ X.float()).double() - Ud @ (Ld[:, None] * (Ud.T @ X)))
        comps = {}
        for q in (0, 1):
            Ur, Dr, Vr = rs.fixed_rank(A, k, p, q, seed=a.seed + 100, prec=rs.RSVD_F32)
            torch.cuda.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            Ur, Dr, Vr = rs.fixed_rank(A, k, p, q, seed=a.seed + 100, prec=rs.RSVD_F32)
            g1.record(stream)
            torch.cuda.synchronize()
            Urd, Drd, Vrd = Ur.double(), Dr.double(), Vr.double()
            # A symmetric: A - U D V^T applied to X, and its transpose, alternate in the power iteration
            est, conv = spectral(lambda X: (A @ X.float()).double() - 0.5 * (
                Urd @ (Drd[:, None] * (Vrd.T @ X)) + Vrd @ (Drd[:, None] * (Urd.T @ X))))
            comps["rsvd_fixed_rank_q%d" % q] = {"value": 1000.0 / g0.elapsed_time(g1), "unit": "solves/s",
                                                "spectral_residual_rel_of_symmetrized": est}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev_tf32
    fma = 2.0 * n * n * l + n * l * l
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    per_ms = ms / a.steps
    achieved = 2.0 * fma / (per_ms / 1000.0) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
            "traffic": None, "algorithmic_flops": 2.0 * fma,
            "kernel": "gemm_simt_kernel (A G and A Q, binary32 SIMT)",
            "peak_source": "152 SMs x 128 binary32 lanes x 2 flops x 2.07 GHz",
            "note": "whole solve time over the two products' FLOPs"}
    cpu = None
    if not a.no_cpu:
        ns = min(a.sample, n)
        As = spd_matrix_np(ns, seed=a.seed)
        t0 = time.perf_counter()
        scaled, reps = 0.0, 0
        while time.perf_counter() - t0 < 10.0 and reps < 20:
            scaled += nystrom_oracle_solve(a, As, a.seed)
            reps += 1
        cpu = {"value": reps / scaled, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": nystrom_sample_text(a, ns, reps, scaled / reps)}
    line = {"metric": METRIC, "value": a.steps / (ms / 1000.0), "unit": "solves/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": per_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": nystrom_name(a),
                       "l2": "inputs larger than L2 (A is %.2f GB; L2 129 MB)" % (n * n * 4 / 1e9)},
            "roofline": roof, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clk,
            "error": {"spectral_residual_rel": ny, "spectral_estimate_last_rel_change": ny_conv,
                      "lambda_k+1_rel(Eckart-Young)": (k + 1) ** -1.5,
                      "max_rel_err_lambda_1..k_vs_construction": float(
                          ((L.cpu() - torch.arange(1, k + 1, dtype=torch.float64).pow(-1.5)).abs()
                           / torch.arange(1, k + 1, dtype=torch.float64).pow(-1.5)).max())},
            "comparators": comps}
    print(json.dumps(line))


# ----------------------------------------------------------- batched -------
BATCH_TOL = 1e-6
BATCH_R = 64
BATCH_B = 16


def batched_name(a):
    return ("batched adaptive: %d fp32 blocks A_ij = 1/|x_i - y_j| (unit-cube clouds 3 apart), m, n ~ U{64..1024}, "
            "tol %g relative Frobenius, b = %d, max rank %d" % (a.count, BATCH_TOL, BATCH_B, BATCH_R))


def batched_oracle_sample(a, seconds, start=0):
    """The float64 oracle's blocked adaptive finder on blocks start, start + 1,
    ... of the same workload (formed on the host), for about `seconds`.
    Returns (blocks solved, seconds, mean m n of the sample)."""
    import numpy as np
    import oracle
    from workloads import kernel_block
    done, t_run, mn = 0, 0.0, 0
    p = start
    while t_run < seconds and done < a.count:
        A = kernel_block(p % a.count, seed=a.seed).astype(np.float64)
        t0 = time.perf_counter()
        oracle.adaptive_blocked(A, BATCH_TOL, b=BATCH_B, seed=a.seed + (p % a.count), max_rank=BATCH_R)
        t_run += time.perf_counter() - t0
        mn += A.shape[0] * A.shape[1]
        done += 1
        p += 1
    return done, t_run, mn / max(done, 1)


def run_batched(a):
    """rsvd_batched on the whole batch per step, replayed from a CUDA graph;
    beside it the plain binary32 single-problem adaptive path on a sample of
    the blocks, and the float64 oracle on a sample on the host cores."""
    import numpy as np
    import torch
    import paper_1607_01649_gb300 as rs
    from workloads import kernel_block_shapes, kernel_block_torch

    world, rank, local = dist_setup(a)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    else:
        dist = None

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    seed = a.seed + 1000 * rank
    shapes = kernel_block_shapes(a.count, seed=seed)
    plan = rs.BatchPlan(shapes, R=BATCH_R, device=dev)
    for p in range(a.count):
        kernel_block_torch(p, plan.block(p), seed=seed)
    h = rs.handle(local)
    side = torch.cuda.Stream(device=dev)
    # the launch variant (loads in flight per thread) is chosen by the
    # library's autotuner on this batch before the graph is captured
    variant, variant_ms = rs.batched_autotune(plan, BATCH_TOL, block=BATCH_B, seed=seed, stream=side)
    side.synchronize()
    with torch.cuda.stream(side):
        for _ in range(a.warmup):
            code = rs.batched_run(plan, BATCH_TOL, block=BATCH_B, seed=seed, stream=side)
            if code != rs.RSVD_OK:
                raise rs.RsvdError(code, rs.last_error(h))
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    launches0 = rs.rsvd_kernel_launches(h)
    with torch.cuda.graph(graph, stream=side):
        code = rs.batched_run(plan, BATCH_TOL, block=BATCH_B, seed=seed, stream=side)
    if code != rs.RSVD_OK:
        raise rs.RsvdError(code, rs.last_error(h))
    launches_per_step = rs.rsvd_kernel_launches(h) - launches0
    graph.replay()
    torch.cuda.synchronize()

    # ---- timed region: K graph replays (inputs 4.9 GB, larger than L2)
    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    with torch.cuda.stream(side):
        ev[0].record(side)
        for i in range(a.steps):
            graph.replay()
            ev[i + 1].record(side)
    barrier()
    clk = clocks.stop()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(a.steps)]
    ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dist, dev)
    value = replica_throughput(world, a.count * a.steps, ms)
    status = plan.status[:a.count].cpu().numpy()
    ranks = plan.rank[:a.count].cpu().numpy().astype(np.int64)
    errs = plan.err[:a.count].cpu().numpy()

    # ---- roofline: the persistent kernel moves A once for ||A||_F and the
    # first sample, then 4 passes of the working copy per block step (read for
    # A_j G, read for Q^T A_j, read and write for the update)
    mn = np.array([m * n for m, n in shapes], dtype=np.float64)
    steps_p = np.ceil(ranks / float(BATCH_B))
    alg_bytes = float(np.sum(4.0 * mn * (1.0 + 4.0 * steps_p)))
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        hbm, peak_src = 6800.0, "fallback"
    per_ms = statistics.median(per)
    achieved = alg_bytes / (per_ms / 1000.0) / 1e9
    # binary32 FMAs: 16 per element for the first sample, then per block step
    # 16 (C), 32 (U1) and 16 + 16 (U2 and the next sample, not after the last)
    fma = float(np.sum(mn * (16.0 + 80.0 * steps_p - 16.0)))
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": batched_traffic(float(mn.sum())), "algorithmic_bytes": alg_bytes,
            "kernel": "batched_kernel (one CTA per problem, persistent, largest-first queue)",
            "avg_ms": per_ms, "peak_source": peak_src,
            "alu": {"achieved_tflops": 2.0 * fma / (per_ms / 1000.0) / 1e12, "peak_tflops": alu_peak,
                    "frac": 2.0 * fma / (per_ms / 1000.0) / 1e12 / alu_peak,
                    "peak_source": "152 SMs x 128 binary32 lanes x 2 flops x 2.07 GHz"},
            "note": "graph replay time (order kernel + persistent kernel)"}

    # ---- e2e: every block copied in from pinned host memory, U, D, V, ranks
    # and residuals copied out, all inside the timed region
    e2e = None
    if not a.no_e2e:
        Ah = torch.empty_like(plan.A, device="cpu").pin_memory()
        Ah.copy_(plan.A)
        Uh = torch.empty_like(plan.U, device="cpu").pin_memory()
        Vh = torch.empty_like(plan.V, device="cpu").pin_memory()
        Dh = torch.empty_like(plan.D, device="cpu").pin_memory()
        rh = torch.empty_like(plan.rank, device="cpu").pin_memory()
        eh = torch.empty_like(plan.err, device="cpu").pin_memory()
        steps_e2e = max(1, min(a.steps, 5))
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(side):
            f0.record(side)
            for i in range(steps_e2e):
                plan.A.copy_(Ah, non_blocking=True)
                rs.batched_run(plan, BATCH_TOL, block=BATCH_B, seed=seed, stream=side)
                for d_, h_ in ((plan.U, Uh), (plan.V, Vh), (plan.D, Dh), (plan.rank, rh), (plan.err, eh)):
                    h_.copy_(d_, non_blocking=True)
            f1.record(side)
        barrier()
        ems = max_over_ranks(f0.elapsed_time(f1), dist, dev)
        nb = lambda t: t.numel() * t.element_size()
        e2e = {"value": replica_throughput(world, a.count * steps_e2e, ems), "unit": "solves/s",
               "h2d_bytes_per_step": nb(plan.A),
               "d2h_bytes_per_step": nb(plan.U) + nb(plan.V) + nb(plan.D) + nb(plan.rank) + nb(plan.err),
               "steps": steps_e2e}
        del Ah, Uh, Vh

    # ---- plain binary32: the single-problem adaptive path (rsvd_adaptive_tol),
    # one call per block, on an evenly spaced sample of the blocks
    f32 = None
    if not a.no_f32:
        idx = list(range(0, a.count, max(1, a.count // 256)))
        for p in idx[:4]:
            rs.adaptive_tol(plan.block(p), BATCH_TOL, block=BATCH_B, max_rank=BATCH_R, seed=seed + p)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record()
        agree = 0
        for p in idx:
            _, D1, _, r1, _, _ = rs.adaptive_tol(plan.block(p), BATCH_TOL, block=BATCH_B, max_rank=BATCH_R,
                                                 seed=seed + p)
            agree += int(r1 == int(ranks[p]))
        g1.record()
        torch.cuda.synchronize()
        f32 = {"value": len(idx) / (g0.elapsed_time(g1) / 1000.0), "unit": "solves/s",
               "sample": "%d evenly spaced blocks, one rsvd_adaptive_tol call each" % len(idx),
               "same_rank_as_batched": agree / float(len(idx))}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None
    cpu = None
    if not a.no_cpu:
        done, t_run, mn_s = batched_oracle_sample(a, 12.0)
        cpu = {"value": done / t_run, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "float64 oracle adaptive_blocked on blocks 0..%d of the workload (mean m n %.0f vs %.0f "
                         "over the batch), %.1f s" % (done - 1, mn_s, float(mn.mean()), t_run)}
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": batched_name(a), "graph": "one CUDA graph replay per step",
                       "autotuned_variant": {"chosen": variant, "rows_cols_ahead": rs.rsvd_batched_variant_info(variant),
                                             "ms_per_variant": variant_ms},
                       "l2": "inputs larger than L2 (%.2f GB of blocks; L2 129 MB)" % (4.0 * mn.sum() / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * a.steps, "clocks": clk,
            "error": {"max_residual_rel": float(errs.max()), "tol": BATCH_TOL,
                      "blocks_converged": int(np.sum(status == 0)), "mean_rank": float(ranks.mean()),
                      "max_rank": int(ranks.max())},
            "plain_f32": f32}
    if dist is not None:
        dist.destroy_process_group()
    return line


def run_reference_batched(a):
    """The oracle arm for the batched workload: each step solves a bounded
    sample of blocks with the float64 oracle on the host cores."""
    world, rank, local = dist_setup(a)
    if rank != 0:
        return
    for w in range(a.warmup):
        batched_oracle_sample(a, 0.5, start=w)
    done, t_run, mn_s = 0, 0.0, 0.0
    for i in range(a.steps):
        d, t, m_ = batched_oracle_sample(a, 10.0 / max(a.steps, 1), start=done)
        done, t_run, mn_s = done + d, t_run + t, mn_s + m_ * d
    value = done / t_run
    sample = ("float64 oracle adaptive_blocked on blocks 0..%d of the workload (mean m n %.0f), about %.1f s per "
              "step" % (done - 1, mn_s / max(done, 1), t_run / a.steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * a.count / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": batched_name(a)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def sub_args(a, workload, steps=5, warmup=2):
    """Arguments of a sub-record of the default run: the workload's own
    defaults, a few steps, no CPU oracle, no e2e, no comparators."""
    import argparse as _ap
    b = _ap.Namespace(**vars(a))
    b.workload = workload
    for key in ("prec", "m", "n", "k", "p", "q", "seed", "sample"):
        setattr(b, key, None)
    b = apply_defaults(b)
    b.steps, b.warmup = steps, warmup
    b.no_cpu = b.no_e2e = b.no_f32 = True
    return b


def compact(line):
    """The figures of a sub-record's line that the default run carries."""
    keep = ("value", "unit", "ms_per_step", "steps", "dtype", "config", "roofline", "error", "clocks",
            "gpu_launches", "variants")
    return {k: line[k] for k in keep if k in line}


def main():
    a = parse()
    if a.workload == "batched":
        if a.impl == "reference":
            run_reference_batched(a)
        else:
            line = run_batched(a)
            if line is not None:
                print(json.dumps(line))
    elif a.workload == "nystrom":
        (run_reference_nystrom if a.impl == "reference" else run_nystrom)(a)
    elif a.workload == "controller":
        (run_reference_controller if a.impl == "reference" else run_controller)(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        line = run_ours(a)
        if line is None:
            return
        if a.workload == "poly" and not a.no_extra and line["n_gpus"] == 1:
            # the other configurations, measured in the same run: the PCA
            # matrix with e4m3 sketches (and implicit centring of the same
            # matrix with column offsets), the batched kernel blocks
            import torch
            extra = {}
            for wl, fn in (("pca", run_ours), ("batched", run_batched)):
                torch.cuda.empty_cache()
                try:
                    sub = fn(sub_args(a, wl))
                    extra[wl] = compact(sub) if sub is not None else None
                except Exception as exc:
                    extra[wl] = {"error": str(exc)[:300]}
            line["extra"] = extra
        print(json.dumps(line))


if __name__ == "__main__":
    main()
