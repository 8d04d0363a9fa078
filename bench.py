"""Benchmark of the GB300 hot path (one JSON line on rank 0).

A step is one pass of the whole crystal hot path over the 32-atom / 8x8x8
workload (96 branches, T = 300 K, sigma = 0.05 THz, 3 sigma):
kald_phonons -> kald_linewidths -> kald_kappa_rta, inputs and outputs
resident on the device.  value = momentum-conserving three-phonon triplets
(N_k^2 nb^3 per step) per second.  `e2e` is the same metric through the same
calls with HOST buffers (host<->device copies inside the timed region).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the linewidths of one q-point per step, plus its phonons), on the
host cores.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import kald_inputs as ki  # noqa: E402

METRIC = "3-phonon triplets/sec (kappa time-to-solution path)"
UNIT = "triplets/s"
WORKLOADS = {"C1": ki.c1, "C2": ki.c2, "C3": ki.c3, "C4": ki.c4, "C5": ki.c5}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_throughput(local_ms: float, world: int, units_per_step: float, steps: int, device=None):
    """Whole-job rate of N replicas (weak scaling, no data-path collective):
    the slowest rank's time (max over ranks) for `steps` steps, and
    world * units_per_step * steps / that time.  The max is one all-reduce on
    `device` (a CUDA device under NCCL, the CPU under gloo)."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * units_per_step * steps / (total_ms / 1e3)


# ------------------------------------------------------------- oracle timing
def time_oracle_sample(w, n_q: int = 1, n_modes: int = 4):
    """Oracle on a bounded sample of the workload: for a crystal, phonons on
    the full mesh + linewidths of n_q q-points (all q', both processes); for a
    Gamma-only system, its phonons + the linewidths of n_modes modes.
    Returns (triplets/s, seconds, description)."""
    from oracle import anharmonic as an
    from oracle import phonons as ph
    s = w.systems[0]
    t0 = time.perf_counter()
    nu, eig = ph.phonons(s, w.mesh)
    if w.n_q == 1:
        nb = s.n_branches
        modes = list(range(nb // 2, nb // 2 + n_modes))
        an.linewidths_gamma_only(s, nu, eig, w.T, w.sigma_thz, w.n_sigma, modes=modes)
        trip = n_modes * nb * nb
        what = f"phonons of system 0 + linewidths of {n_modes} modes ({trip} triplets)"
    else:
        qs = list(range(1, 1 + n_q))
        an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma, q_list=qs)
        trip = n_q * w.n_q * s.n_branches ** 3
        what = f"phonons on the full mesh + linewidths of {n_q} q-point(s) x all q' ({trip} triplets)"
    dt = time.perf_counter() - t0
    return trip / dt, dt, what


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]()
    cores = os.cpu_count()
    for _ in range(args.warmup):
        time_oracle_sample(w)
    vals, secs = [], []
    sample = ""
    for _ in range(args.steps):
        v, dt, sample = time_oracle_sample(w)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.description}", "global_batch": 1,
                       "parallelism": "host cores", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU arm
def run_kald(args):
    import torch
    import paper_2009_01967_gb300 as kk
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kk.load_library()
    w = WORKLOADS[args.workload]()
    if args.mesh:
        w.mesh = tuple(int(x) for x in args.mesh.split(","))
    gamma_only = w.n_q == 1
    s = w.systems[0]
    nq = w.n_q
    nbs = [x.n_branches for x in w.systems]
    nb = nbs[0]
    opt = kk.Options(temperature_K=w.T, sigma_thz=w.sigma_thz, n_sigma=w.n_sigma,
                     precision=args.precision)
    ctx = kk.Context(local)
    stream = torch.cuda.current_stream(dev)
    ctx.set_stream(stream.cuda_stream)
    n_modes = sum(nq * b for b in nbs)
    n_eig = sum(nq * b * b for b in nbs)
    nu = torch.zeros(n_modes, dtype=torch.float64, device=dev)
    eig = torch.zeros(n_eig, dtype=torch.complex128, device=dev)
    gam = torch.zeros(n_modes, dtype=torch.float64, device=dev)
    kap = torch.zeros((len(nbs), 3, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    trip_info = {}
    offs_m = np.cumsum([0] + [nq * b for b in nbs])
    offs_e = np.cumsum([0] + [nq * b * b for b in nbs])

    def phon(nu_t, eig_t):
        for x, sx in enumerate(w.systems):
            kk.kald_phonons(ctx, sx, w.mesh, nu_thz=nu_t[offs_m[x]:offs_m[x + 1]],
                            eigvec=eig_t[offs_e[x]:offs_e[x + 1]], want_vel=False)

    def kappa(nu_t, eig_t, gam_t, kap_t):
        if gamma_only:
            kk.kald_kappa_qhgk(ctx, w.systems, nu_t, eig_t, gam_t, opt, kappa=kap_t)
        else:
            kk.kald_kappa_rta(ctx, s, w.mesh, nu_t, eig_t, gam_t, opt, kappa=kap_t[0])

    def step():
        phon(nu, eig)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, trip = kk.kald_linewidths(ctx, w.systems, w.mesh, nu, eig, opt, gamma=gam)
        ev1.record(stream)
        kappa(nu, eig, gam, kap)
        trip_info["trip"] = trip
        return ev0, ev1

    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = kk.kald_kernel_launches()
    step_ms, lw_ms = [], []
    for _ in range(args.steps):
        flush.fill_(float(_))                      # L2 flush, outside the step events
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e0, e1 = step()
        b.record(stream)
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
        lw_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = kk.kald_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    triplets_step = sum(nq * nq * b ** 3 for b in nbs)
    total_ms, value = job_throughput(float(sum(step_ms)), world, triplets_step, args.steps, device=dev)

    # ---- end to end through host buffers (pinned), same calls
    nu_h = torch.zeros(n_modes, dtype=torch.float64).pin_memory().numpy()
    eig_h = torch.zeros(n_eig, dtype=torch.complex128).pin_memory().numpy()
    gam_h = torch.zeros(n_modes, dtype=torch.float64).pin_memory().numpy()
    kap_h = np.zeros((len(nbs), 3, 3))
    sys_bytes = sum(x.masses.nbytes + x.positions.nbytes + x.fc2_idx.nbytes + x.fc2.nbytes +
                    x.fc3_idx.nbytes + x.fc3.nbytes for x in w.systems)
    e2e_ms = []
    for it in range(0 if args.no_e2e else max(1, min(args.steps, 3))):
        flush.fill_(2.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phon(nu_h, eig_h)
        kk.kald_linewidths(ctx, w.systems, w.mesh, nu_h, eig_h, opt, gamma=gam_h)
        kappa(nu_h, eig_h, gam_h, kap_h)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    h2d = 3 * sys_bytes + 2 * (nu_h.nbytes + eig_h.nbytes) + gam_h.nbytes
    d2h = nu_h.nbytes + eig_h.nbytes + gam_h.nbytes + kap_h.nbytes
    e2e_value = triplets_step / (float(np.mean(e2e_ms)) / 1e3) if e2e_ms else None

    # ---- roofline of the dominant kernel (linewidth projection)
    trip, allowed = trip_info["trip"]
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2 flops
    lw_avg_s = float(np.mean(lw_ms)) / 1e3
    if gamma_only:
        nu_c = nu.cpu().numpy()
        if args.precision == "bf16split":
            # executed tensor work: 3 BF16 MMAs per product; GEMM1 over all
            # 128 x 128 tiles, GEMM2 over the delta-band tiles (upper triangle)
            flops = 0.0
            cut = w.n_sigma * 2 * np.pi * w.sigma_thz
            for x, b in enumerate(nbs):
                om = 2 * np.pi * nu_c[offs_m[x]:offs_m[x + 1]]
                om = np.where(nu_c[offs_m[x]:offs_m[x + 1]] > opt.omega_min_thz, om, 0.0)
                nt = -(-b // 128)
                ld = -(-b // 128) * 128
                lo = np.full(nt, np.inf); hi = np.full(nt, -np.inf)
                for m in range(b):
                    if om[m] > 0:
                        lo[m // 128] = min(lo[m // 128], om[m]); hi[m // 128] = max(hi[m // 128], om[m])
                def band(ww, a, c):
                    return ((ww + lo[a] - hi[c] < cut) and (ww + hi[a] - lo[c] > -cut)) or \
                           ((ww - hi[a] - hi[c] < cut) and (ww - lo[a] - lo[c] > -cut))
                n_tiles = 0
                for ww in om[om > 0]:
                    for a in range(nt):
                        for c in range(a, nt):
                            if hi[a] >= lo[a] and hi[c] >= lo[c] and (band(ww, a, c) or (c != a and band(ww, c, a))):
                                n_tiles += 1
                n_valid = int(np.sum(om > 0))
                flops += 3 * 2.0 * 128 * 128 * ld * (n_valid * nt * nt + n_tiles)
            kernel = "tc_gemm_kernel"
        else:
            # per valid mode: two dense nb^3 contractions (E Y, then (E Y) E^T), 2 flop per FMA
            flops = sum(4.0 * b ** 3 * int(np.sum(nu_c[offs_m[x]:offs_m[x + 1]] > opt.omega_min_thz))
                        for x, b in enumerate(nbs))
            kernel = "g_gemm_nt_kernel"
    else:
        if args.precision == "bf16split":
            # executed tensor work: per pair, GEMM1 and GEMM2 over ceil(nb^2 / 128)
            # row tiles of N = K = 2H (H = nb rounded up to 32); 3 MMAs per
            # product (5 when H <= 64: three-piece eigenvector operand)
            H = -(-nb // 32) * 32
            mt = -(-(nb * nb) // 128)
            n_mma = 5 if H <= 64 else 3
            flops = nq * nq * 2.0 * mt * n_mma * 2.0 * 128 * (2 * H) * (2 * H)
            kernel = "tcx_gemm_kernel"
        else:
            n_valid = int(torch.sum(nu > opt.omega_min_thz).item())
            n_fc3 = s.fc3.shape[0]
            flops = (n_valid * nq * (20.0 * n_fc3 + 8.0 * nb ** 3)     # Y build + T' = eps'^T Y
                     + allowed * 8.0 * nb)                              # phi at delta-allowed pairs
            kernel = "lw_main_kernel"
    achieved = flops / lw_avg_s / 1e12
    timed = ("one kald_linewidths call, CUDA events on its stream: every kernel of the stage "
             "(gather / Y-build, operand splits, GEMMs, reductions), so frac is a lower bound for the "
             "GEMM kernel itself; per-kernel shares are in profiles/")
    if args.precision == "bf16split":
        peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "kernel": kernel, "flops_per_launch": flops,
                    "timed_region": timed,
                    "peak_note": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16, power-capped loop), of measured"}
    else:
        peak = fp32_peak if args.precision == "fp32" else fp32_peak / 64.0
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": kernel, "flops_per_launch": flops, "timed_region": timed,
                    "peak_note": "152 SMs x 128 FP32 lanes x 2 flop x sm_max_mhz" +
                                 ("" if args.precision == "fp32" else " / 64 (FP64)")}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, sample = time_oracle_sample(w)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": sample, "seconds": dt}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "bf16split": "bf16x3"}[args.precision],
                "data": "synthetic",
                "config": {"workload": f"{w.name}: {w.description}", "global_batch": world,
                           "seq_len": None, "parallelism": f"replicas{world}",
                           "l2": "flushed (256 MB write) between timed steps",
                           "precision": args.precision,
                           "linewidth_ms": float(np.mean(lw_ms))},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(launches),      # library kernels in the timed steps (its own counter)
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
                "kappa_W_mK": kap.cpu().numpy().round(6).tolist()[:2],
                "delta_allowed_fraction": allowed / trip}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kald", choices=["kald", "reference"])
    ap.add_argument("--workload", default="C2", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64", "bf16split"],
                    help="default: fp64 for C1 (the plain-method configuration), bf16split (tensor cores) otherwise")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling runs)")
    ap.add_argument("--mesh", default=None, help="override the q-mesh, e.g. 4,4,4 (profiling runs)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp64" if args.workload == "C1" else "bf16split"
    if args.impl == "reference":
        return run_reference(args)
    return run_kald(args)


if __name__ == "__main__":
    sys.exit(main())
