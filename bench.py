"""Benchmark: forward SP2 + adjoint susceptibility at N = 16384 on one GB300.

One step = one full solve of the hot path on a seeded synthetic tight-binding
Hamiltonian (4096 sites x 4 orbitals, N_occ = 8192): the SP2 density of
Eq. DM0 with split-precision (FP16 hi/lo with a 2^11-scaled lo plane, FP32
accumulation) tensor-core products, X_n checkpointed every 4 steps, then the
adjoint recursion of Eq. DM2 seeded with the x-dipole observable,
recomputing each segment of X_n from its checkpoint. Output: D and chi^A.

Prints ONE JSON line (rank 0). Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch one process per GPU with torch.distributed.run; each rank
solves its own seeded problem (independent units, weak scaling, no
collective on the data path; a barrier and a max-reduce of the timings only).

Two further workloads print their own JSON line (one GPU, not run by default):
  --workload fermi  N=8192 gapless spectrum at kT = 0.02 (Sec. V.B): the
                    primal responses to 256 dense H1_k against the dual
                    (one chi^A and 256 contractions), FP16X2 and FP32.
  --workload nonorth  N=8192 non-orthonormal basis (Sec. V.A): the dual weights
                    W_H, W_S once, then three contractions per basis-set
                    dependent perturbation, against one primal response each.
  --workload configs  the other configurations: N=128 microseconds per SP2
                    iteration, N=4096 primal (64 H1) vs dual (4 A) in FP16X2 /
                    FP32 / FP64, N=16384 through torch.autograd vs direct.
  --workload scf    N=4096 tight-binding, 128 site fields: self-consistent
                    response (Eq. DM_CP_SCF) with linear, Anderson and the
                    learned MLP mixer (trained here on 96 fields' linear-mixing
                    trajectories, tested on 32 held-out fields).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N=16384 fwd+adjoint chi: ms, TFLOP/s, %TC peak, rel err vs FP64; mixed vs plain"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gemm_tc_traffic.json")
TC_SOURCE = os.path.join(ROOT, "paper_2409_17033_gb300", "csrc", "gemm_tc.cu")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--ckpt-k", type=int, default=4)
    ap.add_argument("--mode", default="fp16x2")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-resident", action="store_true")
    ap.add_argument("--no-exact", action="store_true",
                    help="skip the accuracy report against the FP64 closed forms (host LAPACK)")
    ap.add_argument("--workload", default="chi",
                    choices=["chi", "fermi", "scf", "nonorth", "configs", "products", "sparse"])
    ap.add_argument("--tau", type=float, default=1e-5, help="block threshold of --workload sparse")
    ap.add_argument("--only", default="all", choices=["all", "config1", "config2", "config3"],
                    help="--workload configs: run one configuration only")
    ap.add_argument("--tiles", default="pair", choices=["pair", "single"],
                    help="product tiles: 256x256 on CTA pairs, or 128x256 on one SM")
    ap.add_argument("--scf-tol", type=float, default=1e-6)
    return ap.parse_args()


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x: float) -> float:
    """Max of x over the ranks (timings: the job takes as long as its slowest rank)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(ws: int, flops_per_rank: float, ms_max: float) -> float:
    """Whole-job throughput: the work all ranks did (each rank solves its own
    problem of the same size) over the slowest rank's time."""
    return ws * flops_per_rank / (ms_max * 1e-3) / 1e12


def workload(n: int, seed: int):
    import workloads
    tb = workloads.tight_binding(n, seed=seed, dtype=np.float32)
    A = workloads.tb_dipole_observables(tb)[0:1].astype(np.float32)  # x-dipole, diagonal
    return tb, A


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def traffic_per_launch(n: int, m: int, k: int):
    """DRAM bytes per product launch from the committed ncu capture, averaged
    over this solve's launch mix (M + M - ceil(M/k) squares, M response
    products), if the capture was taken on the current kernel source and at
    this size; else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    try:
        d = json.load(open(TRAFFIC_FILE))
        src = hashlib.sha256(open(TC_SOURCE, "rb").read()).hexdigest()
        if d.get("kernel_sha256") != src or int(d.get("n", -1)) != n:
            return None
        sq = d["square"]["read_bytes"] + d["square"]["write_bytes"]
        pl = d["plain"]["read_bytes"] + d["plain"]["write_bytes"]
        nsq = m + (m - (m + k - 1) // k)
        return (nsq * sq + m * pl) / (nsq + m)
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.out = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.out = open(os.devnull, "w")
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=self.out, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            txt, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            txt = ""
        rows = []
        for line in txt.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def gpu_uuid():
    try:
        import torch
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def logical_flops(n: int, m: int, k: int) -> float:
    """Logical products of one solve, each 2 N^3: M squares forward, the
    M - ceil(M/k) recomputed squares and M adjoint products Y X (X Y is its
    transpose)."""
    recompute = m - (m + k - 1) // k
    return (m + recompute + m) * 2.0 * float(n) ** 3


def cpu_oracle_sample(n: int, H32: np.ndarray, nocc: float):
    """One SP2 step of the FP64 oracle on an n x n Hamiltonian (one n^3 product), timed."""
    from oracle import sp2 as osp2
    H = H32.astype(np.float64)
    t0 = time.perf_counter()
    osp2.sp2_density(H, nocc, sigma=[1])
    dt = time.perf_counter() - t0
    return dt, 2.0 * float(n) ** 3 / dt / 1e12


def rel_fro(a, b) -> float:
    a = np.asarray(a, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cpu_oracle_accuracy(tb, a_diag: np.ndarray, D_gpu: np.ndarray, chi_gpu: np.ndarray,
                        a1_gpu: np.ndarray, v: np.ndarray) -> dict:
    """The oracle leg's accuracy report: the FP64 closed forms on the host
    (LAPACK eigendecomposition; D = theta(mu I - H), chi^A by Daleckii-Krein,
    a1_k = Tr[chi^A H1_k]) against the solve's outputs, as relative Frobenius
    errors, with the conditioning kappa = spectral width / HOMO-LUMO gap."""
    from oracle import exact
    t0 = time.perf_counter()
    e, V = exact.eigh(tb.H.astype(np.float64))
    kappa = float((e[-1] - e[0]) / (e[tb.nocc] - e[tb.nocc - 1]))
    eD = rel_fro(D_gpu, exact.density_zero_T(e, V, tb.nocc))
    chi_ex = exact.response_zero_T(e, V, tb.nocc, np.diag(a_diag.astype(np.float64)))
    del V
    eC = rel_fro(chi_gpu, chi_ex)
    a1_ex = np.diagonal(chi_ex) @ v.T.astype(np.float64)
    del chi_ex
    return {"D": eD, "chi": eC, "a1": rel_fro(a1_gpu, a1_ex), "kappa": kappa,
            "gap": float(e[tb.nocc] - e[tb.nocc - 1]),
            "a1_perturbations": int(v.shape[0]), "host_s": time.perf_counter() - t0,
            "reference": "FP64 closed forms on the host (LAPACK dsyevd, Daleckii-Krein)"}


def chi_config(args, ws: int) -> dict:
    """The workload of the default line (both arms)."""
    n = args.n
    return {
        "workload": (f"tight-binding N={n} ({n // 4} sites x 4 orbitals, density 0.1, r<6), "
                     f"N_occ={n // 2}: forward SP2 (Eq. DM0) + adjoint chi (Eq. DM2) of the "
                     f"x-dipole, X_n checkpointed every {args.ckpt_k} steps"),
        "n": n, "mode": args.mode, "ckpt_k": args.ckpt_k, "global_batch": ws,
        "parallelism": f"replicas x{ws}",
        "l2": "inputs larger than L2 (each N x N FP32 matrix is 1 GiB at N=16384)",
    }


def run_reference(args, ws, rank):
    """The oracle as it stands on the host cores, on this workload. Each step is
    a bounded sample of the solve: one FP64 oracle SP2 step (one m^3 product,
    m = N/2) on the leading m x m block of the same Hamiltonian, reported as the
    solve's metric (TFLOP/s) at that rate."""
    if rank != 0:
        return
    tb, A = workload(args.n, seed=0)
    m = args.n // 2
    Hs = np.ascontiguousarray(tb.H[:m, :m])
    for _ in range(args.warmup):
        cpu_oracle_sample(m, Hs, m // 2)
    times = []
    for _ in range(args.steps):
        dt, _ = cpu_oracle_sample(m, Hs, m // 2)
        times.append(dt)
    t = sum(times) / len(times)
    val = 2.0 * float(m) ** 3 / t / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": chi_config(args, ws),
        "sample": (f"each step: one FP64 oracle SP2 step (one {m}^3 product) on the leading "
                   f"{m} x {m} block of the N={args.n} Hamiltonian; the solve's flops at that rate"),
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": (f"one FP64 SP2 step ({m}^3 product, {t:.1f} s) per step on the "
                                    f"leading {m} x {m} block; numpy/BLAS, all host threads")},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, ws, rank):
    import torch

    import paper_2409_17033_gb300 as sp2

    dev = torch.cuda.current_device()
    tb, A = workload(args.n, seed=rank)
    n = args.n
    H = torch.from_numpy(tb.H).cuda()
    Ad = torch.from_numpy(A).cuda()
    h = sp2.Handle()
    kw = dict(direction="backward", diag_only=True, mode=args.mode, want_density=True,
              ckpt_k=args.ckpt_k, handle=h)

    def step(timing=False):
        return sp2.sp2_susceptibility(H, tb.nocc, Ad, time_kernels=timing, **kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clk = ClockSampler(gpu_uuid())
    barrier(ws)
    torch.cuda.synchronize()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        chi, D, info = step(timing=True)
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = allmax(ws, ms)
    info = infos[-1]
    M = info["M"]
    lflops = logical_flops(n, M, args.ckpt_k)
    value = whole_job_tflops(ws, lflops, ms_max)
    exec_tflops = info["executed_flops"] / (ms * 1e-3) / 1e12
    pk, pk_kind = peaks()
    # dominant kernel: the tcgen05 product kernel, timed by events around each launch
    prod_ms = statistics.mean(i["product_ms"] for i in infos)
    prod_launch = statistics.mean(i["product_launches_timed"] for i in infos)
    alg = statistics.mean(i["algorithmic_flops"] for i in infos)
    achieved = alg / (prod_ms * 1e-3) / 1e12
    peak = pk["bf16_tflops_sustained"]
    traffic = traffic_per_launch(n, info["M"], args.ckpt_k)
    gpu_launches = sum(i["kernel_launches"] for i in infos)

    quality = {
        "M": M, "trace_err": abs(info["trace"] - tb.nocc), "idem_err": info["idem_err"],
        "product_time_share": prod_ms / ms,
    }
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"{args.mode} (split 16-bit products, f32 accumulate/master)",
        "data": "synthetic",
        "config": chi_config(args, ws),
        "ms_per_solve": ms_max, "tflops_effective": value / ws, "tflops_executed": exec_tflops,
        "tc_peak_frac_executed": exec_tflops / peak,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_gemm_tc (tcgen05 split 16-bit product)",
                     "launches_per_step": prod_launch,
                     "peak_kind": f"bf16_tflops_sustained ({pk_kind})"},
        "quality": quality,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }

    # end to end through the C ABI with host buffers (pinned), copies timed; right
    # after the device-resident timing, so that both see the same thermal state
    if not args.no_e2e:
        Hh = torch.from_numpy(tb.H).pin_memory().numpy()
        Ah = torch.from_numpy(A).pin_memory().numpy()
        hh = sp2.Handle()
        kwh = dict(kw)
        kwh["handle"] = hh
        # page-locked result buffers, as a user streaming results to the host would pass
        kwh["out"] = torch.empty((1, n, n), dtype=torch.float32).pin_memory().numpy()
        kwh["D_out"] = torch.empty((n, n), dtype=torch.float32).pin_memory().numpy()
        sp2.sp2_susceptibility(Hh, tb.nocc, Ah, **kwh)
        barrier(ws)
        ev = [_events() for _ in range(args.steps)]
        clk_e = ClockSampler(clk.gpu_id)
        clk_e.start()
        t0 = time.perf_counter()
        for i in range(args.steps):
            ev[i][0].record(stream)
            chi_h, D_h, _ = sp2.sp2_susceptibility(Hh, tb.nocc, Ah, **kwh)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        clocks_e = clk_e.stop()
        e2e_gpu_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        e2e_s = allmax(ws, e2e_s)
        # raw page-locked copy rates on this machine (torch pinned tensors), for reading
        # the end-to-end overhead
        scratch = torch.empty_like(H)
        hpin = torch.empty(H.shape, dtype=H.dtype).pin_memory()
        torch.cuda.synchronize()
        c0, c1 = _events()
        c0.record(stream)
        scratch.copy_(hpin, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        h2d_ms = c0.elapsed_time(c1)
        c0.record(stream)
        hpin.copy_(scratch, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        d2h_ms = c0.elapsed_time(c1)
        del scratch, hpin
        line["e2e"] = {"value": whole_job_tflops(ws, lflops, e2e_s * 1e3), "unit": "TFLOP/s",
                       "h2d_bytes_per_step": int(Hh.nbytes + Ah.nbytes),
                       "d2h_bytes_per_step": int(chi_h.nbytes + D_h.nbytes),
                       "ms_per_step": e2e_s * 1e3,
                       "gpu_ms_per_step": e2e_gpu_ms,
                       "clocks": clocks_e,
                       "pinned_copy_gbs": {"h2d": Hh.nbytes / (h2d_ms * 1e-3) / 1e9,
                                           "d2h": D_h.nbytes / (d2h_ms * 1e-3) / 1e9}}
        del hh

    # plain forms on the same GPU: per-product timings of the FP32 CUDA-core
    # kernels extrapolated to this solve's product count (stated as such)
    if not args.no_plain and rank == 0:
        try:
            H64 = H
            _, inf_sq = sp2.sp2_density(H64, tb.nocc, mode="fp32", sigma=[1], time_kernels=True,
                                        handle=h)
            _, _, inf_y = sp2.sp2_susceptibility(H64, tb.nocc, Ad, "forward", diag_only=True,
                                                 mode="fp32", sigma=[1], time_kernels=True, handle=h)
            sq_ms = inf_sq["product_ms"]
            y_ms = inf_y["product_ms"] - sq_ms
            rec = M - (M + args.ckpt_k - 1) // args.ckpt_k
            est = (M + rec) * sq_ms + M * max(y_ms, 0.0)
            line["plain_fp32"] = {"ms_per_solve_extrapolated": est,
                                  "tflops_effective": lflops / (est * 1e-3) / 1e12,
                                  "square_ms": sq_ms, "response_product_ms": y_ms,
                                  "note": "FP32 CUDA-core products, per-product event times x product count"}
        except Exception as ex:  # report, do not hide
            line["plain_fp32"] = {"error": str(ex)}
        try:
            _, inf_sq = sp2.sp2_density(H, tb.nocc, mode="fp64", sigma=[1], time_kernels=True,
                                        handle=h)
            _, _, inf_y = sp2.sp2_susceptibility(H, tb.nocc, Ad, "forward", diag_only=True,
                                                 mode="fp64", sigma=[1], time_kernels=True, handle=h)
            sq_ms = inf_sq["product_ms"]
            y_ms = inf_y["product_ms"] - sq_ms
            rec = M - (M + args.ckpt_k - 1) // args.ckpt_k
            est = (M + rec) * sq_ms + M * max(y_ms, 0.0)
            line["plain_fp64"] = {"ms_per_solve_extrapolated": est,
                                  "tflops_effective": lflops / (est * 1e-3) / 1e12,
                                  "square_ms": sq_ms, "response_product_ms": y_ms,
                                  "note": "FP64 CUDA-core products, per-product event times x product count"}
            line["speedup_vs_plain_fp64"] = est / ms
        except Exception as ex:
            line["plain_fp64"] = {"error": str(ex)}
        h.release_history()

    # the same solve with the X_n history sized to device memory (every X_n kept
    # when it fits: no recompute), one timed solve after one warm-up
    if not args.no_resident and rank == 0:
        try:
            kwr = dict(kw)
            kwr["ckpt_k"] = "auto"
            sp2.sp2_susceptibility(H, tb.nocc, Ad, **kwr)
            torch.cuda.synchronize()
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            chi_r, _, inf_r = sp2.sp2_susceptibility(H, tb.nocc, Ad, **kwr)
            r1.record(stream)
            torch.cuda.synchronize()
            rms = r0.elapsed_time(r1)
            kr = inf_r["ckpt_k"]
            line["history_resident"] = {
                "ms_per_solve": rms, "ckpt_k": kr, "M": inf_r["M"],
                "tflops_effective": logical_flops(n, inf_r["M"], kr) / (rms * 1e-3) / 1e12,
                "chi_max_abs_diff_vs_k4": float((chi_r - chi).abs().max()),
                "note": "ckpt_k=auto: smallest checkpoint interval whose history fits in free HBM"}
            del chi_r
            h.release_history()
        except Exception as ex:
            line["history_resident"] = {"error": str(ex)}


    if rank == 0 and ws == 1 and not args.no_exact:
        # accuracy of this solve against the FP64 closed forms (the oracle leg, host LAPACK);
        # a1 over 64 site-potential perturbations, contracted on the device
        import workloads
        v = workloads.tb_site_potentials(tb, 64, seed=1)
        a1 = sp2.response_contract(chi, torch.from_numpy(v.astype(np.float32)).cuda(),
                                   diag_only=True, handle=h)[0].cpu().numpy()
        acc = cpu_oracle_accuracy(tb, A[0], D.cpu().numpy(), chi[0].cpu().numpy(), a1, v)
        line["quality"]["rel_err_vs_exact"] = acc

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        dt, tf = cpu_oracle_sample(n, tb.H, tb.nocc)
        line["cpu_baseline"] = {"value": tf, "unit": "TFLOP/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": (f"one FP64 oracle SP2 step (one N^3 product) at N={n}, "
                                           f"{dt:.1f} s; numpy/BLAS on all host threads"),
                                "ms_per_solve_extrapolated": dt * 1e3 * lflops / (2.0 * n ** 3)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_fermi(args, ws, rank):
    """N=8192, e ~ U[-1, 1] with Haar eigenvectors, kT = 0.02, mu = 0 (Sec. V.B,
    canonical responses, 20 doublings). The 256 perturbations H1_k are
    symmetric with iid N(0, 1/N) upper triangles, drawn on the device by
    torch's Philox generator (seed 1000); the observable A comes from the
    seeded host generator. Primal: D1_k for every k, then Tr[A D1_k]. Dual:
    chi^A once, then Tr[chi^A H1_k] (Eq. Equivalence)."""
    import torch

    import paper_2409_17033_gb300 as sp2
    import workloads
    n, K, kT = 8192, 256, 0.02
    p = workloads.metallic_spectrum(n, k=0, seed=rank)
    H = torch.from_numpy(p.H.astype(np.float32)).cuda()
    A = torch.from_numpy(p.A.astype(np.float32)).cuda()[None]
    del p
    g = torch.Generator(device="cuda")
    g.manual_seed(1000 + rank)
    H1 = torch.empty((K, n, n), dtype=torch.float32, device="cuda")
    for k in range(K):
        x = torch.randn((n, n), generator=g, device="cuda") / np.sqrt(n)
        H1[k] = torch.triu(x) + torch.triu(x, 1).T
    del x
    h = sp2.Handle()
    kw = dict(canonical=True, n_doublings=20, handle=h, time_kernels=True)
    stream = torch.cuda.current_stream()
    out = {}
    for mode in ("fp16x2", "fp32"):
        sp2.sp2_fermi(H, 0.0, kT, A, mode=mode, want_density=False, **kw)   # warm-up
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(stream)
        chi, _, inf_d = sp2.sp2_fermi(H, 0.0, kT, A, mode=mode, want_density=False, **kw)
        a_dual = sp2.response_contract(chi, H1, handle=h)[0]
        e1.record(stream)
        torch.cuda.synchronize()
        out[mode] = {"dual_ms": e0.elapsed_time(e1), "dual_product_ms": inf_d["product_ms"],
                     "dual_alg_flops": inf_d["algorithmic_flops"], "a_dual": a_dual}
        if mode == "fp16x2":
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record(stream)
            D1, _, inf_p = sp2.sp2_fermi(H, 0.0, kT, H1, mode=mode, want_density=False, **kw)
            a_prim = sp2.response_contract(D1, A, handle=h)[:, 0]
            e1.record(stream)
            torch.cuda.synchronize()
            del D1
            out[mode].update(primal_ms=e0.elapsed_time(e1), primal_product_ms=inf_p["product_ms"],
                             primal_alg_flops=inf_p["algorithmic_flops"], a_prim=a_prim)
    pk, pk_kind = peaks()
    m = out["fp16x2"]
    rel = lambda a, b: float((a - b).norm() / b.norm())   # noqa: E731
    achieved = m["primal_alg_flops"] / (m["primal_product_ms"] * 1e-3) / 1e12
    line = {
        "metric": "N=8192 finite-T responses to 256 H1_k: primal vs dual ms; a1 agreement",
        "value": m["primal_ms"] / m["dual_ms"], "unit": "x (primal ms / dual ms)",
        "n_gpus": 1, "higher_is_better": True, "dtype": "fp16x2", "data": "synthetic",
        "config": {"workload": "gapless e~U[-1,1], Haar Q, N=8192, kT=0.02, mu=0, 20 doublings, "
                               "canonical mu_1, 256 dense H1_k (device Philox), 1 observable",
                   "n": n, "K": K},
        "primal_ms": m["primal_ms"], "dual_ms": m["dual_ms"],
        "dual_ms_fp32": out["fp32"]["dual_ms"],
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk["bf16_tflops_sustained"],
                     "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops_sustained"],
                     "kernel": "k_gemm_tc (primal products)",
                     "peak_kind": f"bf16_tflops_sustained ({pk_kind})"},
        "a1_rel_diff": {"primal_vs_dual_fp16x2": rel(m["a_prim"], m["a_dual"]),
                        "dual_fp16x2_vs_dual_fp32": rel(m["a_dual"], out["fp32"]["a_dual"]),
                        "primal_fp16x2_vs_dual_fp32": rel(m["a_prim"], out["fp32"]["a_dual"])},
    }
    print(json.dumps(line), flush=True)


def run_scf(args, ws, rank):
    """Self-consistent response on the N=4096 tight-binding workload (1024
    sites x 4 orbitals) for 128 site fields V_ext ~ N(0, 0.1^2): fields 0..95
    train the learned mixer, fields 96..127 are held out. Mixers: linear
    (alpha 0.3 and 0.7), Anderson, the learned correction on a unit step, and
    Anderson with that learned step as its preconditioner. Responses in FP16X2,
    whose rounding floors the residual near 3e-6 at this size; below 1e-5 every
    mixer continues in BF16X3 responses (24-bit operands, FP32 accumulation) with
    the same SP2 polynomial, to the target residual (1e-6). The residual is the
    plain method's in every case. Kernels: the regularised
    K_ab = 1/sqrt(r_ab^2 + 1) (positive definite) for the mixer comparison,
    and the literal K_ab = 1/r_ab, whose fixed-point map is unstable (linear
    mixing diverges; reported as measured)."""
    import torch

    import paper_2409_17033_gb300 as sp2
    import workloads
    n = 4096
    tb = workloads.tight_binding(n, seed=rank, dtype=np.float32)
    H = torch.from_numpy(tb.H).cuda()
    V = torch.from_numpy(workloads.site_fields(tb, 128, seed=2)).cuda()
    Kreg = torch.from_numpy(workloads.site_kernel(tb, "regularised")).cuda()
    Klit = torch.from_numpy(workloads.site_kernel(tb, "literal")).cuda()
    train, test = V[:96].contiguous(), V[96:].contiguous()
    h = sp2.Handle()
    tol, alpha, mode, floor_tol = args.scf_tol, 0.3, "fp16x2", 1e-5
    stream = torch.cuda.current_stream()

    def timed(**kw):
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(stream)
        r = sp2.sp2_scf_response(H, tb.nocc, 4, mode=mode, handle=h, allow_noconv=True,
                                 return_info=True, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"scf {kw.get('mixer')} fields {kw['Vext'].shape[0]}: {r[2]} iterations, residual "
              f"{r[1][-1]:.2e}, {ms / 1e3:.1f} s", file=sys.stderr, flush=True)
        return r, ms

    # training data: the training fields' solution (Anderson, to the FP16X2 floor) and
    # their unit-step (alpha = 1) linear-mixing trajectories; pairs
    # (r / |r|, (q* - q - r) / |r|). The learned correction rides on a unit step: for
    # q = chi0 (V + K q) it is A (I - A)^-1 r with A = chi0 K, which is concentrated on
    # the few stiff (long-wavelength) modes of A, where a unit step alone oscillates
    a_mlp = 1.0
    (q_star, r_star, it_star, _, _), t_star = timed(K=Kreg, Vext=train, mixer="anderson",
                                                    tol=floor_tol, max_iter=30)
    (_, _, it_tr, (tr, tq), _), t_tr = timed(K=Kreg, Vext=train, mixer="linear", alpha=a_mlp,
                                             tol=floor_tol, max_iter=30, record=True)
    R = tr.reshape(-1, tr.shape[-1])
    T = (q_star[None] - tq - a_mlp * tr).reshape(-1, tq.shape[-1])
    nr = R.norm(dim=1, keepdim=True)
    keep = nr[:, 0] > 0
    X = (R[keep] / nr[keep]).float().contiguous()
    Tn = (T[keep] / nr[keep]).float().contiguous()
    del tr, tq, R, T
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    ns, dh = X.shape[1], 256
    W1 = (torch.randn((dh, ns), generator=g, device="cuda") / np.sqrt(ns)).contiguous()
    W2 = (0.1 * torch.randn((ns, dh), generator=g, device="cuda") / np.sqrt(dh)).contiguous()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = sp2.mlp_train(W1, W2, X, Tn, steps=2000, lr=3e-3, handle=h)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = {}
    refine = "bf16x3"
    mixers = (("linear", dict(mixer="linear", alpha=alpha), 150),
              ("linear_alpha0.7", dict(mixer="linear", alpha=0.7), 80),
              ("anderson", dict(mixer="anderson", alpha=alpha, history=8), 60),
              ("mlp", dict(mixer="mlp", alpha=a_mlp, W1=W1, W2=W2, bf16_infer=True), 80),
              ("anderson_mlp", dict(mixer="anderson_mlp", alpha=a_mlp, history=8, W1=W1, W2=W2,
                                    bf16_infer=True), 60))
    for name, kw, cap in mixers:
        (q, r, it, _, inf), t = timed(K=Kreg, Vext=test, tol=tol, max_iter=cap, refine_mode=refine,
                                      refine_below=floor_tol, **kw)
        res[name] = {"iterations": it, "split_iterations": inf["refine_iter"],
                     "final_residual": float(r[-1]), "ms": t, "converged": bool(r[-1] <= tol),
                     "residuals": [float(x) for x in r], "q": q}
    qa = res["anderson"]["q"]
    for name in res:
        q = res[name].pop("q")
        res[name]["q_rel_diff_vs_anderson"] = float((q - qa).norm() / qa.norm())
    lit = {}
    for name, kw, cap in (("linear", dict(mixer="linear", alpha=alpha), 12),
                          ("anderson", dict(mixer="anderson", alpha=alpha, history=8), 30)):
        (q, r, it, _, _), t = timed(K=Klit, Vext=test, tol=floor_tol, max_iter=cap, **kw)
        lit[name] = {"iterations": it, "final_residual": float(r[-1]), "ms": t,
                     "converged": bool(r[-1] <= floor_tol), "residuals": [float(x) for x in r]}
    line = {
        "metric": f"N=4096 SCF response, 128 fields: iterations to residual {tol:g} (MLP vs linear vs Anderson)",
        "value": res["linear"]["iterations"] / max(res["mlp"]["iterations"], 1),
        "unit": "x (linear alpha=0.3 iterations / MLP iterations, 32 held-out fields)",
        "n_gpus": 1, "higher_is_better": True,
        "dtype": f"fp16x2 responses, {refine} below {floor_tol:g}; MLP fp32 train, bf16 infer",
        "data": "synthetic",
        "config": {"workload": "tight-binding N=4096 (1024 sites x 4), 128 fields V_ext~N(0,0.1^2): "
                               "96 train / 32 held out; MLP 1024->256->1024 ReLU, no biases, "
                               "on a unit linear step",
                   "n": n, "tol": tol, "alpha": alpha, "alpha_mlp": a_mlp,
                   "refine_below": floor_tol, "refine_mode": refine},
        "regularised_K": res, "literal_K": lit,
        "training": {"solution_anderson_iterations": it_star, "solution_residual": float(r_star[-1]),
                     "solution_ms": t_star, "trajectory_iterations": it_tr, "trajectory_ms": t_tr,
                     "pairs": int(X.shape[0]), "adam_steps": 2000, "train_s": t_train,
                     "loss_first": float(hist[0]), "loss_last": float(hist[-1])},
    }
    print(json.dumps(line), flush=True)


def run_nonorth(args, ws, rank):
    """N=8192 non-orthonormal problem (seeded: S = L L^T, H = L H^perp L^T with
    a gapped H^perp, N_occ = 4096; FP16X2). One call gives D, W_H, W_S; then
    a_tau = Tr[A_t D] + Tr[W_H H_t] + Tr[W_S S_t] for 64 dense perturbation
    triples drawn on the device (torch Philox, seed 2000), as three batched
    contractions. The primal form needs one density-matrix response per
    perturbation: one sp2_response of the same size and mode is timed."""
    import torch

    import paper_2409_17033_gb300 as sp2
    import workloads
    n, K = 8192, 64
    p = workloads.nonorth_problem(n, nocc=n // 2, k=0, seed=rank)
    H, S, A = (torch.from_numpy(x.astype(np.float32)).cuda() for x in (p.H, p.S, p.A))
    del p
    h = sp2.Handle()
    stream = torch.cuda.current_stream()
    sp2.sp2_nonorth_susceptibility(H, S, n // 2, A, mode="fp16x2", handle=h)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(stream)
    D, WH, WS, _, info = sp2.sp2_nonorth_susceptibility(H, S, n // 2, A, mode="fp16x2", handle=h)
    e1.record(stream)
    torch.cuda.synchronize()
    setup_ms = e0.elapsed_time(e1)
    g = torch.Generator(device="cuda")
    g.manual_seed(2000 + rank)
    def sym_batch():
        out = torch.empty((K, n, n), dtype=torch.float32, device="cuda")
        for k in range(K):
            x = torch.randn((n, n), generator=g, device="cuda") / np.sqrt(n)
            out[k] = torch.triu(x) + torch.triu(x, 1).T
        return out
    At = sym_batch()
    Ht = sym_batch()
    St = sym_batch()
    for _ in range(2):
        sp2.response_contract(D[None], At, handle=h)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(stream)
    a = (sp2.response_contract(D[None], At, handle=h) + sp2.response_contract(WH[None], Ht, handle=h)
         + sp2.response_contract(WS[None], St, handle=h))[0]
    e1.record(stream)
    torch.cuda.synchronize()
    dual_ms = e0.elapsed_time(e1)
    dual_per_tau = dual_ms / K
    # response_contract roofline: every Q_k read once plus each left factor once
    ctr_bytes = (3 * K + 3) * n * n * 4
    pk, pk_kind = peaks()
    del At, St
    # one primal density-matrix response of the same size and mode (one perturbation)
    sp2.sp2_response(H, n // 2, Ht[0:1], mode="fp16x2", handle=h)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(stream)
    sp2.sp2_response(H, n // 2, Ht[0:1], mode="fp16x2", handle=h)
    e1.record(stream)
    torch.cuda.synchronize()
    primal_per_tau = e0.elapsed_time(e1)
    line = {
        "metric": "N=8192 non-orthonormal dual derivative: setup ms (W_H, W_S) and ms per perturbation, dual vs primal",
        "value": primal_per_tau / dual_per_tau, "unit": "x (primal ms / dual ms per perturbation)",
        "n_gpus": 1, "higher_is_better": True, "dtype": "fp16x2", "data": "synthetic",
        "config": {"workload": "S = L L^T (unit lower-triangular L, overlap 0.5/sqrt(N)), "
                               "H = L H^perp L^T with a gapped H^perp, N=8192, N_occ=4096; "
                               "64 dense perturbation triples (A_t, H_t, S_t)", "n": n, "K": K},
        "setup_ms": setup_ms, "newton_schulz_iterations": info["refine_iter"], "M": info["M"],
        "dual_ms_per_perturbation": dual_per_tau, "primal_ms_per_perturbation": primal_per_tau,
        "breakeven_perturbations": setup_ms / max(primal_per_tau - dual_per_tau, 1e-9),
        "a_tau_finite": bool(torch.isfinite(a).all()),
        "roofline": {"bound": "hbm", "achieved": ctr_bytes / (dual_ms * 1e-3) / 1e9,
                     "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": ctr_bytes / (dual_ms * 1e-3) / 1e9 / pk["hbm_gbs"],
                     "kernel": "k_contract_dense_f32 (3 x 64 contractions)",
                     "peak_kind": f"hbm_gbs ({pk_kind})"},
    }
    print(json.dumps(line), flush=True)


def run_products(args, ws, rank):
    """The two product kernels alone, for kernel timing and profiling: each step
    is one forward response step (sigma = +1) of the x-dipole on the N x N
    tight-binding H (--n, default 16384), i.e. one plain product Y X and one
    square X^2, in that order, with the tiles of --tiles. Per-launch times are
    CUDA events around each product launch (the library's time_kernels)."""
    import numpy as np
    import torch

    import paper_2409_17033_gb300 as sp2
    import workloads
    n = args.n
    tb = workloads.tight_binding(n, seed=0, dtype=np.float32)
    H = torch.from_numpy(tb.H).cuda()
    A = torch.from_numpy(workloads.tb_dipole_observables(tb)[0:1].astype(np.float32)).cuda()
    h = sp2.Handle()
    h.set_option("pair_tiles", 1 if args.tiles == "pair" else 0)
    sq, tot = [], []
    for i in range(args.warmup + args.steps):
        _, _, inf = sp2.sp2_susceptibility(H, n // 2, A, "forward", diag_only=True, mode=args.mode,
                                           sigma=[1], time_kernels=True, handle=h)
        torch.cuda.synchronize()
        _, ind = sp2.sp2_density(H, n // 2, mode=args.mode, sigma=[1], time_kernels=True, handle=h)
        torch.cuda.synchronize()
        if i >= args.warmup:
            tot.append(inf["product_ms"])
            sq.append(ind["product_ms"])
    k = {"bf16x3": 6.0, "fp16x2": 3.0, "bf16x2": 3.0}.get(args.mode, 1.0)   # tensor products each
    sq_ms = float(np.median(sq))
    pl_ms = float(np.median(tot)) - sq_ms
    sq_tf = n * (n + 1) * n * k / sq_ms / 1e9
    pl_tf = 2.0 * n ** 3 * k / pl_ms / 1e9
    line = {"metric": f"N={n} product kernels: algorithmic TFLOP/s per launch (square X^2, plain Y X)",
            "value": pl_tf, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": args.mode, "data": "synthetic",
            "config": {"workload": f"tight-binding N={n}, one forward response step (sigma=+1)",
                       "tiles": args.tiles, "n": n},
            "square": {"ms": sq_ms, "tflops": sq_tf}, "plain": {"ms": pl_ms, "tflops": pl_tf}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sparse(args, ws, rank):
    """Thresholded block-sparse SP2 (Sec. II's thresholded sparse algebra) on the
    gapped periodic tight-binding rod at N = 8192, 16384 and 32768 (--n caps the
    largest): per size the dense FP16X2 solve and the block-sparse one at
    --tau, their times (CUDA events, median of the timed steps), M, the formed
    share of the upper 256 x 256 blocks, and the relative difference of the two
    density matrices. The sparse time per N shows the scaling; value is the
    speedup at the largest N."""
    import numpy as np
    import torch

    import paper_2409_17033_gb300 as sp2
    import workloads
    stream = torch.cuda.current_stream()
    h = sp2.Handle()
    sizes = [n for n in (8192, 16384, 32768) if n <= max(args.n, 8192)]
    rows = {}
    for n in sizes:
        tb = workloads.tight_binding_rod(n, seed=0, dtype=np.float32)
        H = torch.from_numpy(tb.H).cuda()
        tb = None
        res = {}
        for kind in ("dense", "sparse"):
            kw = dict(mode=args.mode, handle=h)
            if kind == "sparse":
                kw["block_tau"] = args.tau
            ts = []
            for i in range(args.warmup + args.steps):
                e0, e1 = _events()
                e0.record(stream)
                D, info = sp2.sp2_density(H, n // 2, **kw)
                e1.record(stream)
                torch.cuda.synchronize()
                if i >= args.warmup:
                    ts.append(e0.elapsed_time(e1))
            res[kind] = (float(np.median(ts)), D, info)
        dd, ds = res["dense"][1], res["sparse"][1]
        rows[n] = {"dense_ms": res["dense"][0], "sparse_ms": res["sparse"][0],
                   "speedup": res["dense"][0] / res["sparse"][0],
                   "M_dense": res["dense"][2]["M"], "M_sparse": res["sparse"][2]["M"],
                   "block_fill": res["sparse"][2]["block_fill"],
                   "rel_diff_D": float(torch.linalg.norm(ds - dd) / torch.linalg.norm(dd)),
                   "trace_err": abs(res["sparse"][2]["trace"] - n / 2),
                   "executed_tflops_sparse": res["sparse"][2]["executed_flops"] / (res["sparse"][0] * 1e9)}
        del H, dd, ds, res
        torch.cuda.empty_cache()
    top = sizes[-1]
    line = {"metric": f"block-sparse SP2 density: speedup over the dense solve at N={top}",
            "value": rows[top]["speedup"], "unit": "x", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": args.mode,
            "data": "synthetic",
            "config": {"workload": "periodic tight-binding rod (density 0.1, width 6, r<6, stagger 2.0), "
                                   "sites sorted along the rod, N_occ=N/2",
                       "tau": args.tau, "block": 256, "sizes": sizes},
            "sizes": {str(k): v for k, v in rows.items()}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_configs(args, ws, rank):
    """The other configurations of the metric as measurement lines (one GPU):
    config 1, N=128 gapped random spectrum (FP64 to idem_tol 1e-10, and FP16X2):
    ms per solve and microseconds per SP2 iteration of the density, the backward
    susceptibility and the 8 responses; config 2, N=4096 tight binding: the primal
    form (64 site-potential responses, then Tr[A_l D1_k]) against the dual form
    (chi of the 4 observables, then Tr[chi_l H1_k]) in FP16X2, FP32 and FP64 (FP64
    extrapolated from per-product event times); config 3, N=16384: the forward
    SP2 + adjoint through torch.autograd (SP2Density, dense incoming gradient)
    beside the direct backward susceptibility call."""
    import torch

    import paper_2409_17033_gb300 as sp2
    import workloads
    stream = torch.cuda.current_stream()
    h = sp2.Handle()

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        e0, e1 = _events()
        e0.record(stream)
        r = None
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    out = {"config1": {}, "config2": {}, "config3": {}}
    # ---------------------------------------------------------------- config 1
    if args.only in ("all", "config1"):
        p = workloads.random_spectrum(128, nocc=64, k=8, seed=0)
        for mode, dt in (("fp64", torch.float64), ("fp16x2", torch.float32)):
            H = torch.from_numpy(p.H).to(dt).cuda()
            A = torch.from_numpy(p.A[None]).to(dt).cuda()
            H1 = torch.from_numpy(p.H1).to(dt).cuda()
            kw = dict(mode=mode, handle=h, idem_tol=1e-10 if mode == "fp64" else 0.0)
            t_d, (_, inf) = timed(lambda: sp2.sp2_density(H, p.nocc, **kw), reps=20)
            t_c, _ = timed(lambda: sp2.sp2_susceptibility(H, p.nocc, A, "backward", **kw), reps=20)
            t_r, _ = timed(lambda: sp2.sp2_response(H, p.nocc, H1, **kw), reps=20)
            m = inf["M"]
            out["config1"][mode] = {"M": m, "density_ms": t_d, "density_us_per_iteration": 1e3 * t_d / m,
                                    "backward_chi_ms": t_c, "responses8_ms": t_r,
                                    "responses8_us_per_iteration": 1e3 * t_r / m}
    # ---------------------------------------------------------------- config 2
    if args.only in ("all", "config2"):
        tb = workloads.tight_binding(4096, seed=0, dtype=np.float32)
        A4 = workloads.tb_dipole_observables(tb)                  # (4, N) diagonals
        v = workloads.tb_site_potentials(tb, 64, seed=1)         # (64, N) diagonals
        for mode, dt in (("fp16x2", torch.float32), ("fp32", torch.float32), ("fp64", torch.float64)):
            H = torch.from_numpy(tb.H).to(dt).cuda()
            Ad = torch.from_numpy(A4).to(dt).cuda()
            vd = torch.from_numpy(v).to(dt).cuda()
            if mode != "fp64":
                def primal():
                    D1, _, inf = sp2.sp2_response(H, tb.nocc, vd, diag_only=True, mode=mode, handle=h)
                    return sp2.response_contract(D1, Ad, diag_only=True, handle=h), inf
                def dual():
                    chi, _, inf = sp2.sp2_susceptibility(H, tb.nocc, Ad, "backward", diag_only=True,
                                                         mode=mode, handle=h)
                    return sp2.response_contract(chi, vd, diag_only=True, handle=h), inf
                t_p, (a_p, inf_p) = timed(primal)
                t_q, (a_q, inf_q) = timed(dual)
                a_p = a_p.cpu().numpy().T      # (4, 64)
                a_q = a_q.cpu().numpy()
                out["config2"][mode] = {"M": inf_q["M"], "primal_ms": t_p, "dual_ms": t_q,
                                        "primal_over_dual": t_p / t_q,
                                        "a1_primal_vs_dual": float(np.linalg.norm(a_p - a_q) / np.linalg.norm(a_q))}
            else:
                # one square and one 64-response step (fixed branch), event-timed, times the
                # product counts of this mode's converged run (M from a density solve)
                _, inf_d = sp2.sp2_density(H, tb.nocc, mode="fp64", idem_tol=1e-10, handle=h)
                m = inf_d["M"]
                _, inf_s = sp2.sp2_density(H, tb.nocc, mode="fp64", sigma=[1], time_kernels=True, handle=h)
                _, _, inf_y = sp2.sp2_response(H, tb.nocc, vd, diag_only=True, mode="fp64", sigma=[1],
                                               time_kernels=True, handle=h)
                _, _, inf_a = sp2.sp2_susceptibility(H, tb.nocc, Ad, "forward", diag_only=True,
                                                     mode="fp64", sigma=[1], time_kernels=True, handle=h)
                sq = inf_s["product_ms"]
                y64 = inf_y["product_ms"] - sq
                y4 = inf_a["product_ms"] - sq
                rec = m - (m + 3) // 4
                out["config2"][mode] = {"M": m, "primal_ms_extrapolated": m * (sq + y64),
                                        "dual_ms_extrapolated": (m + rec) * sq + m * y4,
                                        "primal_over_dual": m * (sq + y64) / ((m + rec) * sq + m * y4),
                                        "note": "per-product event times x product counts"}
            del H
    # ---------------------------------------------------------------- config 3
    if args.only in ("all", "config3"):
        n = 16384
        tb3, A3 = workload(n, seed=0)
        H = torch.from_numpy(tb3.H).cuda()
        a = torch.from_numpy(A3[0]).cuda()
        Ad = torch.from_numpy(A3).cuda()
        hh = sp2.Handle()

        def via_autograd():
            Hg = H.clone().requires_grad_(True)
            D = sp2.sp2_density_autograd(Hg, tb3.nocc, mode="fp16x2", ckpt_k=4, handle=hh)
            loss = (D.diagonal() * a).sum()          # Tr[A D], A the x-dipole
            loss.backward()
            return Hg.grad

        def direct():
            chi, _, _ = sp2.sp2_susceptibility(H, tb3.nocc, Ad, "backward", diag_only=True,
                                               mode="fp16x2", ckpt_k=4, handle=hh)
            return chi[0]

        t_a, g = timed(via_autograd)
        t_b, chi = timed(direct)
        out["config3"] = {"autograd_ms": t_a, "direct_ms": t_b,
                          "grad_vs_direct_chi_max_abs": float((g - chi).abs().max()),
                          "chi_max_abs": float(chi.abs().max()),
                          "note": "autograd: forward SP2 (keep_history, k=4), dense incoming gradient "
                                  "diag(A) of Tr[A D], adjoint (Eq. DM2); direct: the diagonal A"}
    line = {"metric": "configs 1-3: N=128 us per SP2 iteration; N=4096 primal vs dual; "
                      "N=16384 autograd vs direct", "n_gpus": 1, "data": "synthetic", **out}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = (1, 0, 0)
    if args.impl == "reference":
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, ws, rank)
        return
    ws, rank, local = dist_setup()
    if args.workload == "fermi":
        run_fermi(args, ws, rank)
    elif args.workload == "nonorth":
        run_nonorth(args, ws, rank)
    elif args.workload == "scf":
        run_scf(args, ws, rank)
    elif args.workload == "configs":
        run_configs(args, ws, rank)
    elif args.workload == "products":
        run_products(args, ws, rank)
    elif args.workload == "sparse":
        run_sparse(args, ws, rank)
    else:
        run_ours(args, ws, rank)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
