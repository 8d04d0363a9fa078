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
    """Whole-job rate: the slowest rank's time (max over ranks, one all-reduce
    on `device`: a CUDA device under NCCL, the CPU under gloo) for `steps`
    steps, and units_per_step * steps / that time, where units_per_step counts
    the units ALL ranks process in one step."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, units_per_step * steps / (total_ms / 1e3)


def inversion_classes(mesh) -> list:
    """The q-points of a Gamma-centred mesh (flat index (k0 m1 + k1) m2 + k2)
    grouped into the pairs {q, -q} (one member where -q = q), ordered by
    their lower index."""
    m0, m1, m2 = (int(x) for x in mesh)
    out = []
    for q in range(m0 * m1 * m2):
        k0, k1, k2 = q // (m1 * m2), (q // m2) % m1, q % m2
        qn = (((m0 - k0) % m0) * m1 + (m1 - k1) % m1) * m2 + (m2 - k2) % m2
        if qn >= q:
            out.append([q] if qn == q else [q, qn])
    return out


def shard_plan(mesh, n_sys: int, world: int, rank: int) -> dict:
    """How rank `rank` of `world` takes its share of one workload (strong
    scaling: the workload is fixed).  A crystal: a contiguous run of the
    inversion classes {q, -q} (ceil(classes / world) each), so that every
    rank's q list is closed under q -> -q and kald_linewidths_qlist projects
    each class once, every q' over the whole mesh; then one all-gather of gamma
    (gather_q_sharded).  Several Gamma-only systems: every world-th system, no
    collective (independent problems).  One Gamma-only system: a replica (its
    modes are not split)."""
    nq = int(np.prod(mesh))
    if world == 1:
        return {"kind": "whole"}
    if nq > 1:
        cls = inversion_classes(mesh)
        per = -(-len(cls) // world)
        lists = [[q for c in cls[r * per:(r + 1) * per] for q in c] for r in range(world)]
        return {"kind": "qlist", "q": lists[rank], "lists": lists, "per": max(len(x) for x in lists)}
    if n_sys >= world:
        return {"kind": "systems", "idx": list(range(rank, n_sys, world))}
    return {"kind": "replica"}


def orbit_pairs(mesh) -> int:
    """Number of orbits of ordered momentum triples (q1, q2, -(q1 + q2)) under
    the six permutations and inversion q -> -q: the projections the tensor
    path makes when Phi3 is symmetric under permutations (host counting)."""
    m = np.asarray(mesh, dtype=np.int64)
    nq = int(np.prod(m))
    k = np.stack(np.meshgrid(*[np.arange(x) for x in m], indexing="ij"), -1).reshape(-1, 3)

    def flat(v):
        v = np.mod(v, m)
        return (v[..., 0] * m[1] + v[..., 1]) * m[2] + v[..., 2]
    q1, q2 = np.meshgrid(np.arange(nq), np.arange(nq), indexing="ij")
    q1, q2 = q1.ravel(), q2.ravel()
    q3 = flat(-(k[q1] + k[q2]))
    neg = flat(-k)
    code = lambda a, b, c: (a * nq + b) * nq + c
    t = code(q1, q2, q3)
    lowest = np.ones(t.shape, dtype=bool)
    for a, b, c in ((q1, q2, q3), (q1, q3, q2), (q2, q1, q3), (q2, q3, q1), (q3, q1, q2), (q3, q2, q1)):
        lowest &= t <= code(a, b, c)
        lowest &= t <= code(neg[a], neg[b], neg[c])
    return int(np.sum(lowest))


def projected_pairs(mesh, plan: dict, opt, nb: int) -> int:
    """(q, q') projections per step on this rank: one per orbit of momentum
    triples on the BF16-split tensor path over the whole mesh (Phi3 of a pair
    potential is symmetric under permutations); else the inversion classes
    {q, -q} of its q-points times the mesh (time reversal, when symmetry is not
    "none" and degenerate averaging is on); else its q-points times the mesh."""
    nq = int(np.prod(mesh))
    qs = plan["q"] if plan["kind"] == "qlist" else list(range(nq))
    if nq == 1 or opt.symmetry == "none" or not opt.degen_tol_thz > 0:
        return len(qs) * nq
    if (opt.symmetry == "all" and opt.precision == "bf16split" and 65 <= nb <= 96
            and plan["kind"] != "qlist"):
        return orbit_pairs(mesh)
    mine = set(qs)
    return sum(1 for c in inversion_classes(mesh) if mine.intersection(c)) * nq


def gather_q_sharded(local, plan: dict, nb: int, nq: int, world: int):
    """All-gather of the q-sharded gamma: `local` holds this rank's
    len(plan["q"]) * nb values (row j = q-point plan["q"][j]); every rank gets
    the full [nq * nb] vector (each rank's rows placed at its q-points)."""
    import torch
    import torch.distributed as dist
    per = plan["per"]
    buf = torch.zeros(per * nb, dtype=local.dtype, device=local.device)
    buf[:local.numel()] = local
    out = torch.empty(world * per * nb, dtype=local.dtype, device=local.device)
    dist.all_gather_into_tensor(out, buf)
    rows = out.view(world * per, nb)
    src = torch.tensor([r * per + j for r in range(world) for j in range(len(plan["lists"][r]))],
                       device=local.device)
    dst = torch.tensor([q for lst in plan["lists"] for q in lst], device=local.device)
    full = torch.empty(nq, nb, dtype=local.dtype, device=local.device)
    full[dst] = rows[src]
    return full.view(-1)


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


# ------------------------------------------------------------- roofline
# DRAM traffic per launch of the dominant kernels from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), scaled to the launch shape
# the benchmark times; the summaries under profiles/ give the command.  None
# when the kernel has changed since the counters were taken.
TRAFFIC_PER_PAIR = {
    # tcx_gemm_kernel on the 32-atom cell, 4x4x4 mesh, one projection per orbit,
    # 38-pair launches: GEMM1 274.37 + 221.41 MB, GEMM2 (three-position
    # epilogue) 274.43 + 4.98 MB (ncu --set full of the first batch's kernels)
    "tcx_gemm1": 495.78e6 / 38,
    "tcx_gemm2": 279.41e6 / 38,
}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of tcx_gemm_kernel on the same cell with a "
                  "4x4x4 mesh (38-pair launches, one projection per orbit), per pair, scaled to the pairs of the "
                  "timed launches")


def _gamma_only_band_tiles(om, cut, tile=128, symmetric=True):
    """Delta-band (tm, tn) tiles of every valid mode, as the library lists them."""
    b = len(om)
    nt = -(-b // tile)
    lo = np.full(nt, np.inf)
    hi = np.full(nt, -np.inf)
    for m in range(b):
        if om[m] > 0:
            lo[m // tile] = min(lo[m // tile], om[m])
            hi[m // tile] = max(hi[m // tile], om[m])

    def band(ww, a, c):
        return ((ww + lo[a] - hi[c] < cut) and (ww + hi[a] - lo[c] > -cut)) or \
               ((ww - hi[a] - hi[c] < cut) and (ww - lo[a] - lo[c] > -cut))
    n_tiles = 0
    for ww in om[om > 0]:
        for a in range(nt):
            for c in range(a if symmetric else 0, nt):
                if hi[a] >= lo[a] and hi[c] >= lo[c] and (band(ww, a, c) or (symmetric and c != a and band(ww, c, a))):
                    n_tiles += 1
    return n_tiles


def roofline_of(args, w, nbs, nu_c, opt, prof, steps, allowed, pairs_step=None):
    """Roofline line of the dominant kernel: ALGORITHMIC work per launch
    (the method's flops, not the split-precision emulation) over the mean
    launch duration from the library's per-launch CUDA events.  `pairs_step`
    is the number of (q, q') projections this rank makes per step."""
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s, FMA = 2 flops
    nq = w.n_q
    s = w.systems[0]
    nb = nbs[0]
    offs = np.cumsum([0] + [nq * b for b in nbs])
    gamma_only = nq == 1
    small = (not gamma_only) and nb <= 6
    executed = None
    if args.precision == "bf16split" and not small:
        if gamma_only:
            names = ("tc_gemm1", "tc_gemm2")
            kernel = "tc_gemm_kernel (GEMM1 T = E Y, GEMM2 delta-band phi tiles + epilogue)"
            cut = w.n_sigma * 2 * np.pi * w.sigma_thz
            alg, exe = 0.0, 0.0
            for x, b in enumerate(nbs):
                nu_x = nu_c[offs[x]:offs[x + 1]]
                om = np.where(nu_x > opt.omega_min_thz, 2 * np.pi * nu_x, 0.0)
                n_valid = int(np.sum(om > 0))
                n_tiles = _gamma_only_band_tiles(om, cut)
                nt, ld = -(-b // 128), -(-b // 128) * 128
                alg += n_valid * 2.0 * b ** 3 + n_tiles * 2.0 * 128 * 128 * b
                exe += 3 * 2.0 * 128 * 128 * ld * (n_valid * nt * nt + n_tiles)
            alg_note = ("per valid mode 2 nb^3 (T = E Y) plus 2 x 128 x 128 x nb per delta-band tile of "
                        "phi = T E^T; executed: 3 BF16 MMAs per product on 128-padded tiles")
        else:
            names = ("tcx_gemm1", "tcx_gemm2")
            kernel = "tcx_gemm_kernel (GEMM1 T' = eps'^T Y_s, GEMM2 phi = T' conj(eps'') + delta epilogue)"
            H = -(-nb // 32) * 32
            mt = -(-(nb * nb) // 128)
            n_mma = 5 if H <= 64 else 3
            alg = nq * nq * 2 * 8.0 * nb ** 4              # two complex nb^4 contractions per pair
            exe = nq * nq * 2.0 * mt * n_mma * 2.0 * 128 * (2 * H) * (2 * H)
            alg_note = ("two dense complex contractions of nb^4 per momentum-conserving pair (8 flop per "
                        "complex MAC); executed: 3 BF16 MMAs per product (5 when nb <= 64)")
        peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
        bound, peak_note = "tensor", ("MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16 in a power-capped "
                                      "loop; the kernels run inside a seconds-long step), of measured")
        executed = exe
    elif small:
        names = ("small_nb",)
        kernel = "sn_kernel (one- and two-atom cells: phase sum, both contractions and the epilogue in registers)"
        n_valid = int(np.sum(nu_c > opt.omega_min_thz))
        n_fc3 = s.fc3.shape[0]
        alg = n_valid * nq * (108.0 * n_fc3 + 8.0 * nb ** 3) + allowed * 8.0 * nb
        alg_note = "per (mode, q'): 108 n_fc3 (phase-summed first-index contraction) + 8 nb^3 (T'), 8 nb per allowed phi"
        peak = fp32_peak if args.precision != "fp64" else fp32_peak / 64.0
        bound, peak_note = "alu", "152 SMs x 128 FP32 lanes x 2 flop x sm_max_mhz" + ("" if args.precision != "fp64" else " / 64 (FP64)")
    else:
        names = ("lw_main",) if not gamma_only else ()
        kernel = "lw_main_kernel" if not gamma_only else "g_gemm_nt_kernel"
        n_valid = int(np.sum(nu_c > opt.omega_min_thz))
        n_fc3 = s.fc3.shape[0]
        if gamma_only:
            alg = sum(4.0 * b ** 3 * int(np.sum(nu_c[offs[x]:offs[x + 1]] > opt.omega_min_thz))
                      for x, b in enumerate(nbs))
        else:
            alg = n_valid * nq * (20.0 * n_fc3 + 8.0 * nb ** 3) + allowed * 8.0 * nb
        alg_note = "Y build + T' per (mode, q'), phi at delta-allowed pairs"
        peak = fp32_peak if args.precision == "fp32" else fp32_peak / 64.0
        bound, peak_note = "alu", "152 SMs x 128 FP32 lanes x 2 flop x sm_max_mhz" + ("" if args.precision == "fp32" else " / 64 (FP64)")
    ms = sum(prof.get(n, (0.0, 0))[0] for n in names)
    launches = sum(prof.get(n, (0.0, 0))[1] for n in names)
    if ms <= 0 or launches == 0:
        return {"bound": bound, "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": kernel, "note": "no timed launches of this kernel"}
    share = (pairs_step / (nq * nq)) if pairs_step is not None else 1.0
    alg *= share
    if executed is not None:
        executed *= share
    alg_per_launch = alg * steps / launches
    mean_s = ms / launches / 1e3
    achieved = alg_per_launch / mean_s / 1e12
    out = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": None, "kernel": kernel, "launches_timed": launches, "mean_launch_ms": mean_s * 1e3,
           "flops_per_launch": alg_per_launch, "algorithmic_work": alg_note, "peak_note": peak_note,
           "timed_region": "CUDA events around every launch of the kernel on its own stream, over the timed steps"}
    if executed is not None:
        exe_per_launch = executed * steps / launches
        out["executed_flops_per_launch"] = exe_per_launch
        out["tensor_pipe_frac"] = exe_per_launch / mean_s / 1e12 / peak
    if not gamma_only and nb == 96 and all(n in TRAFFIC_PER_PAIR for n in names):
        # bytes per launch: per-pair DRAM traffic of each kernel x the pairs all its launches covered
        pairs = share * nq * nq * steps
        out["traffic"] = sum(TRAFFIC_PER_PAIR[n] * pairs for n in names) / launches
        out["traffic_source"] = TRAFFIC_SOURCE
        out["traffic_note"] = ("A1 (Y) and T1 (T') as BF16 hi/lo in HBM: 7.1 MB per pair each way; the "
                               "method's own data (eps, Phi3, gamma) is ~0.1 GB per step")
    other = {n: {"ms": v[0], "launches": v[1]} for n, v in prof.items() if v[1]}
    out["per_kernel_ms"] = other
    return out


def kappa_time_to_solution(kk, ctx, w, opt, phon, kappa, n_modes, n_eig, nbs):
    """kappa from host inputs to host kappa (kald_phonons + kald_linewidths +
    kald_kappa_*): the configured split path, the same path with time reversal
    as its only symmetry (the projections the FP64 path makes; timed after one
    untimed call that tunes its schedule), and the plain FP64 GPU path (time
    reversal); wall time of each and the split kappas' relative errors."""
    import dataclasses
    res = {}
    kaps = {}
    runs = (("split", dataclasses.replace(opt)),
            ("split_inversion", dataclasses.replace(opt, symmetry="inversion")),
            ("fp64", dataclasses.replace(opt, precision="fp64", symmetry="inversion")))
    for name, o in runs:
        for rep in range(2 if name == "split_inversion" else 1):
            nu_h = np.zeros(n_modes)
            eig_h = np.zeros(n_eig, dtype=np.complex128)
            gam_h = np.zeros(n_modes)
            kap_h = np.zeros((len(nbs), 3, 3))
            t0 = time.perf_counter()
            phon(nu_h, eig_h)
            kk.kald_linewidths(ctx, w.systems, w.mesh, nu_h, eig_h, o, gamma=gam_h)
            kappa(nu_h, eig_h, gam_h, kap_h, o)
            res[name] = time.perf_counter() - t0
            kaps[name] = kap_h
    b = kaps["fp64"]
    err = float(np.max(np.abs(kaps["split"] - b)) / np.max(np.abs(b)))
    err_i = float(np.max(np.abs(kaps["split_inversion"] - b)) / np.max(np.abs(b)))
    return {"split_s": res["split"], "fp64_s": res["fp64"], "speedup": res["fp64"] / res["split"],
            "kappa_rel_err_vs_fp64": err, "tolerance": 1e-4, "within_tolerance": err <= 1e-4,
            "split_inversion_only_s": res["split_inversion"],
            "speedup_same_projections": res["fp64"] / res["split_inversion"],
            "kappa_rel_err_inversion_only": err_i,
            "symmetry": {"split": opt.symmetry, "split_inversion_only": "inversion", "fp64": "inversion"},
            "path": "host inputs -> kald_phonons -> kald_linewidths -> kald_kappa -> host kappa"}


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
    units_step = float(sum(w.n_q * w.n_q * x.n_branches ** 3 for x in w.systems))   # whole job
    shard = shard_plan(w.mesh, len(w.systems), world, rank)
    if shard["kind"] == "systems":
        w.systems = [w.systems[x] for x in shard["idx"]]
    elif shard["kind"] == "replica":
        units_step *= world
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
        if gamma_only and len(w.systems) > 1:      # every supercell in one launch sequence
            kk.kald_phonons_batch(ctx, w.systems, nu_thz=nu_t, eigvec=eig_t)
            return
        for x, sx in enumerate(w.systems):
            kk.kald_phonons(ctx, sx, w.mesh, nu_thz=nu_t[offs_m[x]:offs_m[x + 1]],
                            eigvec=eig_t[offs_e[x]:offs_e[x + 1]], want_vel=False)

    def kappa(nu_t, eig_t, gam_t, kap_t, o=None):
        o = o or opt
        if gamma_only:
            kk.kald_kappa_qhgk(ctx, w.systems, nu_t, eig_t, gam_t, o, kappa=kap_t)
        else:
            kk.kald_kappa_rta(ctx, s, w.mesh, nu_t, eig_t, gam_t, o, kappa=kap_t[0])

    def step():
        phon(nu, eig)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        if shard["kind"] == "qlist":
            loc = gam[:len(shard["q"]) * nb]
            trip = (0, 0)
            if shard["q"]:
                _, trip = kk.kald_linewidths_qlist(ctx, s, w.mesh, nu, eig, opt, shard["q"], gamma=loc)
            gam.copy_(gather_q_sharded(loc.clone(), shard, nb, nq, world))
        else:
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
    ctx.profile(True)                              # per-launch CUDA events on the launching streams
    launches0 = kk.kald_kernel_launches()
    step_ms, lw_ms, ph_ms, kp_ms = [], [], [], []
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
        ph_ms.append(a.elapsed_time(e0))
        kp_ms.append(e1.elapsed_time(b))
    torch.cuda.synchronize()
    launches = kk.kald_kernel_launches() - launches0
    prof = ctx.profile_read()
    ctx.profile(False)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    triplets_step = sum(nq * nq * b ** 3 for b in nbs)
    total_ms, value = job_throughput(float(sum(step_ms)), world, units_step, args.steps, device=dev)

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
        if shard["kind"] == "qlist":
            loc = np.zeros(len(shard["q"]) * nb)
            if shard["q"]:
                kk.kald_linewidths_qlist(ctx, s, w.mesh, nu_h, eig_h, opt, shard["q"], gamma=loc)
            full = gather_q_sharded(torch.from_numpy(loc).to(dev), shard, nb, nq, world)
            gam_h[:] = full.cpu().numpy()
        else:
            kk.kald_linewidths(ctx, w.systems, w.mesh, nu_h, eig_h, opt, gamma=gam_h)
        kappa(nu_h, eig_h, gam_h, kap_h)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    if world > 1 and e2e_ms:
        _, e2e_rate = job_throughput(float(sum(e2e_ms)), world, units_step, len(e2e_ms), device=dev)
    else:
        e2e_rate = units_step / (float(np.mean(e2e_ms)) / 1e3) if e2e_ms else None
    h2d = 3 * sys_bytes + 2 * (nu_h.nbytes + eig_h.nbytes) + gam_h.nbytes
    d2h = nu_h.nbytes + eig_h.nbytes + gam_h.nbytes + kap_h.nbytes
    e2e_value = e2e_rate

    # ---- roofline of the dominant kernel, timed per launch inside the steps
    trip, allowed = trip_info["trip"]
    pairs_step = projected_pairs(w.mesh, shard, opt, nbs[0])
    roofline = roofline_of(args, w, nbs, nu.cpu().numpy(), opt, prof, args.steps, allowed, pairs_step)

    # ---- kappa time-to-solution: split path against the plain FP64 GPU path
    tts = None
    if rank == 0 and world == 1 and not args.no_tts and args.precision != "fp64":
        tts = kappa_time_to_solution(kk, ctx, w, opt, phon, kappa, n_modes, n_eig, nbs)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, sample = time_oracle_sample(w)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": sample, "seconds": dt}
    # strong scaling (one fixed workload shared by the ranks) unless a single
    # Gamma-only system runs as replicas
    one_system_gamma = (w.n_q == 1 and shard["kind"] in ("whole", "replica") and len(w.systems) == 1)
    scaling = "weak" if one_system_gamma else "strong"
    parallelism = {"whole": "single GPU", "qlist": f"q-sharded over {world} GPUs (inversion classes), all-gather of gamma (NCCL)",
                   "systems": f"systems dealt over {world} GPUs", "replica": f"replicas{world}"}[shard["kind"]]
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": scaling, "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "bf16split": "bf16x3"}[args.precision],
                "data": "synthetic",
                "config": {"workload": f"{w.name}: {w.description}",
                           "global_batch": 1 if scaling == "strong" else world,
                           "seq_len": None, "parallelism": parallelism,
                           "l2": "flushed (256 MB write) between timed steps",
                           "precision": args.precision,
                           "symmetry": opt.symmetry,
                           "projected_pairs_per_step": (
                               sum(projected_pairs(w.mesh, dict(shard, q=lst), opt, nbs[0]) for lst in shard["lists"])
                               if shard["kind"] == "qlist" else pairs_step),
                           "momentum_pairs_per_step": nq * nq if not gamma_only else None,
                           "linewidth_ms": float(np.mean(lw_ms)),
                           "phonons_ms": float(np.mean(ph_ms)), "kappa_ms": float(np.mean(kp_ms))},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(launches),      # library kernels in the timed steps (its own counter)
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
                "kappa_time_to_solution": tts,
                "kappa_W_mK": kap.cpu().numpy().round(6).tolist()[:2],
                "delta_allowed_fraction": allowed / trip if trip else None}
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
    ap.add_argument("--no-tts", action="store_true",
                    help="skip the kappa time-to-solution comparison with the plain FP64 GPU path")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp64" if args.workload == "C1" else "bf16split"
    if args.impl == "reference":
        return run_reference(args)
    return run_kald(args)


if __name__ == "__main__":
    sys.exit(main())
