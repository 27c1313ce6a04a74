"""Benchmark of the batched FP64 local Hamiltonian (one JSON line on rank 0).

Workload (the configuration the orbital-applications/s metric is quoted on):
192 orbitals in one autotuned, graph-captured plan -- 64 orbitals on each of
three periodic cells with coarse grids 56^3, 48^3 and 40^3 (fine 112^3, 96^3,
80^3), 8 wavelet components per coarse point, FP64, each cell with its own
Gaussian-sum potential, occupations 2.0.  One step = the whole hot path
(uncompress, synthesis, magic filter, V psi + density + Epot, transposed
magic filter, kinetic + Ekin, analysis, compress, reductions) over all 192
orbitals.  The orbitals (1.43 GB per array) exceed the 129 MB L2, so no
flush is needed between steps.

--impl reference times the FP64 CPU oracle (test infrastructure, plain
numpy) on a bounded sample of the same workload (one orbital of each cell per
step) on the host cores.

Multi-GPU (torchrun): every rank runs its own 192 orbitals of the same three
cells (weak scaling, the paper's orbital distribution), and each step ends
with the one exchange that distribution needs: the density (FP64, per cell)
and the energy sums all-reduced over the ranks; value = all ranks' orbitals /
max-over-ranks time.
"""
from __future__ import annotations

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

SIZES = [(56, 56, 56), (48, 48, 48), (40, 40, 40)]
PER_CELL = 64
CFG = 2
METRIC = "H_loc|psi> orbital-applications/s (FP64, batched uneven cells)"
UNIT = "orbital-applications/s"


def workload(per_cell):
    gb = sum(per_cell * 8 * a * b * c for a, b, c in SIZES) * 8 / 1e9
    return {
        "workload": f"batched FP64 local Hamiltonian + density, {3 * per_cell} orbitals: "
                    f"{per_cell} each on periodic coarse 56^3, 48^3, 40^3 cells (fine 112^3, "
                    "96^3, 80^3), 8 components, Gaussian-sum V per cell, occ 2.0; "
                    "autotuned, graph-captured",
        "orbitals": 3 * per_cell,
        "fine_points_per_step": sum(per_cell * 8 * a * b * c for a, b, c in SIZES),
        "l2": f"inputs larger than L2 ({gb:.2f} GB per orbital array), no flush",
    }


WORKLOAD = workload(PER_CELL)
# FP32 HBM bytes per orbital point: the fused chain and the transposing passes
FUSED_BPP, PASSES_BPP = 52.0, 140.0
# FP32 FMAs per orbital point (either chain)
FP32_FMA_PER_POINT = 279.0
# Algorithmic flops per fine point of one kinetic pass: the 29-tap filter of
# Eq. (kinetic1d), one multiply-add per tap; the kernels apply the 27 taps
# above FP64 resolution (the a_{+-14} edge taps are 6.9e-18)
KIN_TAPS_ALGORITHMIC, KIN_TAPS_APPLIED = 29, 27
# Pipe peaks (TFLOP/s, 2 flops per FMA).  Nominal GB300 figures; replaced by
# the FMA-chain probe's measurement (wvl_fma_peak) at the start of each run.
FP64_PEAK_NOMINAL, FP32_PEAK_NOMINAL = 1.25, 80.6
FP64_PEAK_TFLOPS, FP32_PEAK_TFLOPS = FP64_PEAK_NOMINAL, FP32_PEAK_NOMINAL
PEAK_SOURCE = "nominal (probe not run)"


def _measured_hbm_gbs(default=6758.5):
    """Copy bandwidth measured on this GPU type (MEASURED_PEAKS.json beside
    this file), else the value it held when this file was written."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return default


HBM_GBS = _measured_hbm_gbs()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_first_orbital(rank, per_rank):
    """Weak scaling: rank r owns orbitals r * per_rank .. (r + 1) * per_rank - 1
    of the synthetic stream (disjoint, no data shared between ranks)."""
    return rank * per_rank


def max_over_ranks(times, dist, world, device="cpu"):
    """The slowest rank's times (timing is the only cross-rank exchange)."""
    if world <= 1:
        return list(times)
    import torch
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def sum_over_ranks(tensors, dist, world):
    """The one exchange of the orbital distribution (Sec. "Parallel
    distribution"): every rank's density, and its energy sums, added over the
    ranks in place (NCCL on GPU ranks, gloo on CPU ranks); a no-op on one rank."""
    if world <= 1:
        return
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)


def job_throughput(norb_per_rank, world, steps, ms):
    """Whole-job orbital applications per second over all ranks."""
    return norb_per_rank * world * steps / (ms * 1e-3)


def make_inputs(rank, per_cell=PER_CELL):
    from paper_0904_1543_gb300 import inputs
    cell_of_orb = [c for c in range(3) for _ in range(per_cell)]
    first = rank_first_orbital(rank, len(cell_of_orb))
    psi = np.concatenate([inputs.orbital(CFG, first + o, SIZES[c])
                          for o, c in enumerate(cell_of_orb)])
    Vs = [inputs.gaussian_potential(CFG, c, SIZES[c]) for c in range(3)]
    occ = np.full(len(cell_of_orb), 2.0)
    return cell_of_orb, psi, Vs, occ


# ---------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_pipe_peaks(W, gpu_id):
    """FP64 and FP32 FMA-chain rates of this GPU, measured now by the
    library's probe (wvl_fma_peak), with the SM clocks sampled meanwhile;
    they become the roofline denominators of this run."""
    global FP64_PEAK_TFLOPS, FP32_PEAK_TFLOPS, PEAK_SOURCE
    clocks = Clocks(gpu_id)
    clocks.start()
    f64, ms64 = W.fma_peak(W.WVL_F64, 0.3)
    f32, ms32 = W.fma_peak(W.WVL_F32, 0.3)
    clk = clocks.stop()
    FP64_PEAK_TFLOPS, FP32_PEAK_TFLOPS = f64, f32
    PEAK_SOURCE = "measured in this run: FMA-chain probe (wvl_fma_peak), best of 3 launches"
    return {"fp64_tflops": f64, "fp32_tflops": f32, "fp64_ms": ms64, "fp32_ms": ms32,
            "fp64_nominal": FP64_PEAK_NOMINAL, "fp32_nominal": FP32_PEAK_NOMINAL,
            "clocks": clk,
            "how": "8 independent FMA chains per thread (FP32: packed pairs) on every SM, "
                   "about 0.3 s per launch, CUDA events"}


# ---------------------------------------------------------- CPU oracle
def oracle_sample(cell_of_orb, psi, Vs, occ, offsets, norb_per_cell=1):
    """Times the oracle on norb_per_cell orbitals of each cell; returns
    (orbitals, seconds)."""
    import oracle.wavelet as O
    t0 = time.perf_counter()
    done = 0
    for c in range(3):
        idx = [o for o, cc in enumerate(cell_of_orb) if cc == c][:norb_per_cell]
        for o in idx:
            O.hpsi_local(psi[offsets[o]:offsets[o + 1]], Vs[c], occ[o], SIZES[c])
            done += 1
    return done, time.perf_counter() - t0


def _oracle_task(task):
    """One orbital of one cell through the oracle in a worker process: inputs
    from the seeded generators (not timed), then the timed oracle call."""
    import oracle.wavelet as O
    from paper_0904_1543_gb300 import inputs
    c, o = task
    psi = inputs.orbital(CFG, o, SIZES[c])
    V = inputs.gaussian_potential(CFG, c, SIZES[c])
    t0 = time.perf_counter()
    O.hpsi_local(psi, V, 2.0, SIZES[c])
    return time.perf_counter() - t0


def oracle_all_cores(seconds=10.0):
    """The oracle on every host core: one spawned worker process per core,
    each taking orbitals of the three cells in turn (every worker single
    threaded).  Returns (orbital-applications/s, workers, orbitals)."""
    import multiprocessing as mp
    n = max(1, os.cpu_count() or 1)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    times = []
    with ctx.Pool(n) as pool:
        pool.map(_oracle_task, [(2, o) for o in range(n)])      # start-up, not timed
        t0 = time.perf_counter()
        r = 0
        while time.perf_counter() - t0 < seconds:
            times += pool.map(_oracle_task, [((r + w) % 3, w) for w in range(n)])
            r += 1
    return n * len(times) / sum(times), n, len(times)


def offsets_of(cell_of_orb):
    off = [0]
    for c in cell_of_orb:
        off.append(off[-1] + 8 * int(np.prod(SIZES[c])))
    return off


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cell_of_orb, psi, Vs, occ = make_inputs(0)
    off = offsets_of(cell_of_orb)
    for _ in range(args.warmup):
        oracle_sample(cell_of_orb, psi, Vs, occ, off)
    done, secs = 0, 0.0
    for _ in range(args.steps):
        d, s = oracle_sample(cell_of_orb, psi, Vs, occ, off)
        done += d
        secs += s
    value = done / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, sample="one orbital of each cell per step (3 orbitals)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "one orbital of each of the 56^3/48^3/40^3 cells per step, "
                                   "FP64 numpy oracle, single thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_0904_1543_gb300 as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    # a non-default stream: plan graphs are captured and replayed on it
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        _run_ours(args, W, torch, dist, rank, world, local, dev)
    if world > 1:
        dist.destroy_process_group()


def _time_steps(torch, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_variants(args, W, torch, dev):
    """The FP32 batched form (256 orbitals, coarse 48^3) with its error
    against the FP64 oracle and its speedup over the FP64 GPU form, and the
    autograd form (512 orbitals, coarse 64^3, FP32 forward + backward)."""
    import oracle.wavelet as O
    from paper_0904_1543_gb300 import inputs
    out = {}
    # ---- FP32 batched, coarse 48^3 x 256 orbitals
    n = (48, 48, 48)
    g = W.Grid(n)
    norb = 256
    psi64 = inputs.orbitals_device(3, norb, n, dev)
    V64 = torch.from_numpy(inputs.gaussian_potential(3, 0, n)).to(dev)
    occ = torch.full((norb,), 2.0, dtype=torch.float64, device=dev)
    psi32, V32 = psi64.float(), V64.float()
    res = {}
    chains = {}
    for name, p, v, prec, chain in (("f32", psi32, V32, W.WVL_F32, None),
                                    ("f32_passes", psi32, V32, W.WVL_F32, "passes"),
                                    ("f64", psi64, V64, W.WVL_F64, None),
                                    ("emu", psi64, V64, W.WVL_F64_EMU, None)):
        plan = W.Plan([g], [0] * norb, prec=prec, graph=True, autotune=True, chain=chain)
        hp = torch.empty_like(p)
        ek = torch.empty(norb, dtype=torch.float64, device=dev)
        ep = torch.empty_like(ek)
        rho = [torch.zeros(g.fine, dtype=torch.float64, device=dev)]
        plan.autotune(p, [v], occ, hpsi=hp, rho=rho)
        ms = _time_steps(torch, lambda: plan.hpsi(p, [v], occ, hpsi=hp, rho=rho, ekin=ek,
                                                  epot=ep), args.steps, 3)
        rho[0].zero_()
        plan.hpsi(p, [v], occ, hpsi=hp, rho=rho, ekin=ek, epot=ep)
        torch.cuda.synchronize()
        res[name] = (ms, hp, ek, ep, rho[0])
        chains[name] = [ln for ln in plan.describe().splitlines() if ln.startswith("chain:")][0][7:]
        del plan
    ms32, hp32, ek32, ep32, rho32 = res["f32"]
    ms32p = res["f32_passes"][0]
    pts32 = norb * 8 * n[0] * n[1] * n[2]
    # HBM bytes per orbital-point the chain moves: the five fused plane/column
    # kernels 52 B (4 B per element: 8 / 12 / 8 / 12 / 12 per kernel), the 15
    # transposing passes 140 B (4 B in and out per pass; the kinetic passes
    # also carry K and G, 44 B); the potential, density partials and their
    # reduction add under 1 B per orbital-point at 256 orbitals per cell
    fused = chains["f32"].startswith("fused")
    bpp = FUSED_BPP if fused else PASSES_BPP
    ms64, hp64, ek64, ep64, rho64 = res["f64"]
    mse, hpe, eke, epe, rhoe = res["emu"]
    # oracle on two sampled orbitals (FP64 arithmetic on the FP32-rounded inputs)
    Vh = V32.double().cpu().numpy()
    err_h, err_e = 0.0, 0.0
    for o in (0, norb - 1):
        ph = psi32[o].double().cpu().numpy()
        r = O.hpsi_local(ph, Vh, 2.0, n)
        err_h = max(err_h, float(np.abs(hp32[o].double().cpu().numpy() - r["hpsi_c"]).max()
                                 / np.abs(r["hpsi_c"]).max()))
        err_e = max(err_e, abs(float(ek32[o]) - r["ekin"]) / abs(r["ekin"]),
                    abs(float(ep32[o]) - r["epot"]) / abs(r["epot"]))
    # density over all 256 orbitals against the FP64 GPU form (which matches
    # the oracle to 1e-12 in the parity tests)
    err_rho = float((rho32 - rho64).abs().max() / rho64.abs().max())
    # orbital scalar products of the FP32 orbitals in compressed form, FP64
    # products and accumulation: the whole 256 x 256 overlap (symmetric path:
    # the 36 upper 32 x 32 tiles) and <psi_o|H psi_o>
    length = 8 * n[0] * n[1] * n[2]
    ms_ov = _time_steps(torch, lambda: W.overlap(psi32), max(2, args.steps // 3), 2)
    Sov = W.overlap(psi32).cpu().numpy()
    ms_dot = _time_steps(torch, lambda: W.dot(psi32, hp32), args.steps, 2)
    dh = W.dot(psi32, hp32).cpu().numpy()
    ov_err = 0.0
    for i, j in ((0, 0), (0, norb - 1), (17, 130), (norb - 1, norb - 1)):
        a_i = psi32[i].double().cpu().numpy()
        a_j = psi32[j].double().cpu().numpy()
        ref = O.scalar_products(a_i[None], a_j[None])[0, 0]
        ov_err = max(ov_err, abs(Sov[i, j] - ref) / np.sqrt(np.dot(a_i, a_i) * np.dot(a_j, a_j)))
    tiles = (norb + 31) // 32
    dfma = tiles * (tiles + 1) // 2 * 1024 * length
    scalar_products = {
        "overlap_ms": ms_ov, "dot_ms": ms_dot,
        "overlap_fp64_tflops": 2.0 * dfma / (ms_ov * 1e-3) / 1e12,
        "overlap_frac_of_fp64_peak": 2.0 * dfma / (ms_ov * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
        "overlap_rel_err_vs_oracle": float(ov_err),
        "overlap_symmetric": bool(np.array_equal(Sov, Sov.T)),
        "dot_psi_hpsi_vs_ekin_plus_epot": float(np.max(np.abs(dh - (ek32 + ep32).cpu().numpy())
                                                      / np.abs((ek32 + ep32).cpu().numpy()))),
        "what": "S = <psi_i|psi_j> for all 256 FP32 orbitals (FP64 products and sums; 36 "
                "upper 32 x 32 tiles of FP64 FMAs), and <psi_o|H psi_o> per orbital; error: "
                "4 sampled entries against the oracle's correctly rounded sums, relative to "
                "sqrt(<psi_i|psi_i> <psi_j|psi_j>)",
    }
    out["fp32_batched"] = {
        "workload": "256 orbitals, periodic coarse 48^3 (fine 96^3), FP32 convolutions, "
                    "FP64 reductions, one autotuned graph-captured plan",
        "scalar_products": scalar_products,
        "value": norb / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32,
        "chain": chains["f32"],
        "fp32_passes_same_workload": {"value": norb / (ms32p * 1e-3), "ms_per_step": ms32p},
        "fp64_same_workload": {"value": norb / (ms64 * 1e-3), "ms_per_step": ms64},
        "speedup_over_fp64": ms64 / ms32,
        "roofline": {"bound": "hbm", "achieved": bpp * pts32 / (ms32 * 1e-3) / 1e9,
                     "peak": HBM_GBS, "unit": "GB/s",
                     "frac": bpp * pts32 / (ms32 * 1e-3) / 1e9 / HBM_GBS,
                     "bytes_per_orbital_point": bpp,
                     "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"},
        "rel_err_hpsi_vs_oracle": err_h, "rel_err_energies_vs_oracle": err_e,
        "rel_err_rho_vs_fp64_gpu": err_rho,
        "error_sample": "H psi and energies: orbitals 0 and 255 against the FP64 oracle; "
                        "rho: all 256 orbitals against the FP64 GPU form",
    }
    # FP64-accurate tensor-core form: oracle on the same two orbitals (FP64
    # inputs), and every orbital against the native FP64 form
    Vd = V64.cpu().numpy()
    emu_h, emu_e = 0.0, 0.0
    for o in (0, norb - 1):
        r = O.hpsi_local(psi64[o].cpu().numpy(), Vd, 2.0, n)
        emu_h = max(emu_h, float(np.abs(hpe[o].cpu().numpy() - r["hpsi_c"]).max()
                                 / np.abs(r["hpsi_c"]).max()))
        emu_e = max(emu_e, abs(float(eke[o]) - r["ekin"]) / abs(r["ekin"]),
                    abs(float(epe[o]) - r["epot"]) / abs(r["epot"]))
    out["fp64_emu_batched"] = {
        "workload": "256 orbitals, periodic coarse 48^3 (fine 96^3), FP64 arrays; every "
                    "convolution sum on the FP16 tensor cores (six 10-bit digits per operand, "
                    "exact FP32 partial sums, 64-bit recombination), one graph-captured plan",
        "value": norb / (mse * 1e-3), "unit": UNIT, "ms_per_step": mse,
        "speedup_over_fp64": ms64 / mse,
        "rel_err_hpsi_vs_oracle": emu_h, "rel_err_energies_vs_oracle": emu_e,
        "rel_diff_hpsi_vs_fp64_gpu": float((hpe - hp64).abs().max() / hp64.abs().max()),
        "rel_diff_rho_vs_fp64_gpu": float((rhoe - rho64).abs().max() / rho64.abs().max()),
        "error_sample": "oracle: orbitals 0 and 255; FP64 GPU form: all 256 orbitals",
        "timeouts": W.wait_timeouts(),
    }
    del res, hp32, hp64, hpe, psi32
    # ---- preconditioner: 5 PCG iterations of the Helmholtz equation, FP64,
    # the same 256 orbitals of coarse 48^3 (eps_o in [-1.5, -0.2])
    eps = -torch.linspace(0.2, 1.5, norb, dtype=torch.float64, device=dev)
    ncg = 5
    ms_pc = _time_steps(torch, lambda: W.precondition(psi64, eps, g, ncg), max(2, args.steps // 3), 2)
    pts = norb * 8 * n[0] * n[1] * n[2]
    # FP64-pipe work per CG iteration and fine point: synthesis 48 + kinetic 87
    # + analysis 48 DFMA (vector updates are memory-bound and not counted)
    out["precond_fp64"] = {
        "workload": "Helmholtz preconditioner (Eq. precon), 5 PCG iterations per orbital, "
                    "256 orbitals on periodic coarse 48^3, FP64",
        "value": norb / (ms_pc * 1e-3), "unit": "orbitals preconditioned/s (5 iterations)",
        "ms_per_step": ms_pc,
        "fp64_tflops": 2.0 * 183 * pts * ncg / (ms_pc * 1e-3) / 1e12,
        "checked": "tests/test_gpu_precond.py: PCG iterates against the oracle (1e-11)",
    }
    del psi64
    # ---- localisation regions: 64 orbitals on the periodic 48^3 cell, each
    # stored on a ball of radius 20 (scaling) / 10 (wavelets) coarse points
    nr = 64
    occr = torch.full((nr,), 2.0, dtype=torch.float64, device=dev)
    regions = []
    for rc, rf in ((20.0, 10.0), (12.0, 6.0), (8.0, 5.0)):
        cm, fm = inputs.sphere_masks(n, (24, 24, 24), rc, rf)
        reg = W.Region(g, cm, fm)
        pr = inputs.vectors_device(5, nr, reg.clen, dev)
        ms_r = _time_steps(torch, lambda: W.hpsi_local_region(pr, V64, occr, g, reg), 3, 2)
        regions.append({"coarse_radius": rc, "fine_radius": rf,
                        "stored_fraction": reg.clen / (8 * n[0] * n[1] * n[2]),
                        "bounding_box": list(reg.len),
                        "value": nr / (ms_r * 1e-3), "unit": UNIT, "ms_per_step": ms_r})
    out["region_fp64"] = {
        "workload": "local Hamiltonian on region-compressed orbitals, 64 orbitals on a periodic "
                    "coarse 48^3 cell, coarse and fine regions balls of the radii below, FP64; "
                    "along axes where the region's bounding box leaves >= 15 coarse points to "
                    "the cell the chain runs on that box",
        "value": regions[0]["value"], "unit": UNIT, "ms_per_step": regions[0]["ms_per_step"],
        "stored_fraction": regions[0]["stored_fraction"],
        "by_region_size": regions,
        "checked": "tests/test_gpu_region.py (1e-12 against the oracle)",
    }
    # ---- free boundary conditions: 64 orbitals on a 32^3 box (padded cell 48^3)
    nb = (32, 32, 32)
    gb = W.Grid(nb)
    pf = inputs.orbitals_device(6, nr, nb, dev)
    Vf = torch.from_numpy(inputs.gaussian_potential(6, 0, tuple(v + 2 * W.FREE_PAD for v in nb))).to(dev)
    ms_f = _time_steps(torch, lambda: W.hpsi_local_free(pf, Vf, occr, gb), 3, 2)
    # the same 64 orbitals on the periodic 32^3 cell (the box without padding)
    Vp32 = torch.from_numpy(inputs.gaussian_potential(6, 0, nb)).to(dev)
    ms_p32 = _time_steps(torch, lambda: W.hpsi_local(pf, Vp32, occr, gb), 3, 2)
    out["free_bc_fp64"] = {
        "workload": "local Hamiltonian with free boundary conditions, 64 orbitals on a coarse "
                    "32^3 box; every 1D pass on the support its stage needs (fine extents "
                    "64 + 16 for s, y, K and z, 64 + 29 for psi_r), FP64",
        "value": nr / (ms_f * 1e-3), "unit": UNIT, "ms_per_step": ms_f,
        "periodic_same_box": {"value": nr / (ms_p32 * 1e-3), "ms_per_step": ms_p32},
        "cost_vs_periodic": ms_f / ms_p32,
        "checked": "tests/test_gpu_free.py (1e-12 against the free-space oracle)",
    }
    del pr, pf
    torch.cuda.empty_cache()
    # ---- the tensor-core FP64 form on the headline workload (the three cells
    # of `value`), with the oracle on one orbital of each cell
    cell_of_orb, psi_h, Vs_h, occ_h = make_inputs(0, args.per_cell)
    cells = [W.Grid(sz) for sz in SIZES]
    plan = W.Plan(cells, cell_of_orb, prec=W.WVL_F64_EMU, graph=True)
    psi = torch.from_numpy(psi_h).to(dev)
    Vd = [torch.from_numpy(v).to(dev) for v in Vs_h]
    occd = torch.from_numpy(occ_h).to(dev)
    hp = torch.empty_like(psi)
    ek = torch.empty(len(cell_of_orb), dtype=torch.float64, device=dev)
    ep = torch.empty_like(ek)
    rho = [torch.zeros(c.fine, dtype=torch.float64, device=dev) for c in cells]
    ms_h = _time_steps(torch, lambda: plan.hpsi(psi, Vd, occd, hpsi=hp, rho=rho, ekin=ek,
                                                epot=ep), args.steps, 3)
    torch.cuda.synchronize()
    offs = plan.offsets
    eh, ee = 0.0, 0.0
    for c in range(3):
        o = c * args.per_cell
        r = O.hpsi_local(psi_h[offs[o]:offs[o + 1]], Vs_h[c], 2.0, SIZES[c])
        got = hp[offs[o]:offs[o + 1]].cpu().numpy()
        eh = max(eh, float(np.abs(got - r["hpsi_c"]).max() / np.abs(r["hpsi_c"]).max()))
        ee = max(ee, abs(float(ek[o]) - r["ekin"]) / abs(r["ekin"]),
                 abs(float(ep[o]) - r["epot"]) / abs(r["epot"]))
    out["fp64_emu_headline_workload"] = {
        "workload": WORKLOAD["workload"].replace("batched FP64", "batched FP64 (tensor-core "
                                                 "emulated convolutions)"),
        "value": len(cell_of_orb) / (ms_h * 1e-3), "unit": UNIT, "ms_per_step": ms_h,
        "rel_err_hpsi_vs_oracle": eh, "rel_err_energies_vs_oracle": ee,
        "error_sample": "the first orbital of each cell against the FP64 oracle",
        "timeouts": W.wait_timeouts(),
    }
    del plan, psi, hp, rho, Vd
    torch.cuda.empty_cache()
    # ---- the FP32 form on the headline workload: the autotuner's chain and
    # the transposing passes, the oracle (FP64 on the FP32-rounded inputs) on
    # the first orbital of each cell
    psi32_h = psi_h.astype(np.float32)
    Vs32_h = [v.astype(np.float32) for v in Vs_h]
    psi = torch.from_numpy(psi32_h).to(dev)
    Vd = [torch.from_numpy(v).to(dev) for v in Vs32_h]
    hp = torch.empty_like(psi)
    rho = [torch.zeros(c.fine, dtype=torch.float64, device=dev) for c in cells]
    f32 = {}
    for chain in (None, "passes"):
        plan = W.Plan(cells, cell_of_orb, prec=W.WVL_F32, graph=True, autotune=True, chain=chain)
        plan.autotune(psi, Vd, occd, hpsi=hp, rho=rho)
        ms_c = _time_steps(torch, lambda: plan.hpsi(psi, Vd, occd, hpsi=hp, rho=rho, ekin=ek,
                                                    epot=ep), args.steps, 3)
        torch.cuda.synchronize()
        f32[chain] = (ms_c, [ln for ln in plan.describe().splitlines()
                             if ln.startswith("chain:")][0][7:])
        if chain is None:
            eh, ee = 0.0, 0.0
            for c in range(3):
                o = c * args.per_cell
                r = O.hpsi_local(psi32_h[offs[o]:offs[o + 1]].astype(np.float64),
                                 Vs32_h[c].astype(np.float64), 2.0, SIZES[c])
                got = hp[offs[o]:offs[o + 1]].double().cpu().numpy()
                eh = max(eh, float(np.abs(got - r["hpsi_c"]).max() / np.abs(r["hpsi_c"]).max()))
                ee = max(ee, abs(float(ek[o]) - r["ekin"]) / abs(r["ekin"]),
                         abs(float(ep[o]) - r["epot"]) / abs(r["epot"]))
        del plan
    ms_a, chain_a = f32[None]
    pts_h = WORKLOAD["fine_points_per_step"]
    bpp = FUSED_BPP if chain_a.startswith("fused") else PASSES_BPP
    out["fp32_headline_workload"] = {
        "workload": WORKLOAD["workload"].replace("batched FP64", "batched FP32 convolutions "
                                                 "(FP64 reductions)"),
        "value": len(cell_of_orb) / (ms_a * 1e-3), "unit": UNIT, "ms_per_step": ms_a,
        "chain": chain_a,
        "passes_same_workload": {"value": len(cell_of_orb) / (f32["passes"][0] * 1e-3),
                                 "ms_per_step": f32["passes"][0]},
        "roofline": {"bound": "hbm", "achieved": bpp * pts_h / (ms_a * 1e-3) / 1e9,
                     "peak": HBM_GBS, "unit": "GB/s",
                     "frac": bpp * pts_h / (ms_a * 1e-3) / 1e9 / HBM_GBS,
                     "bytes_per_orbital_point": bpp,
                     "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"},
        "roofline_fp32_pipe": {"bound": "alu", "achieved": 2 * FP32_FMA_PER_POINT * pts_h
                               / (ms_a * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                               "unit": "TFLOP/s",
                               "frac": 2 * FP32_FMA_PER_POINT * pts_h / (ms_a * 1e-3) / 1e12
                               / FP32_PEAK_TFLOPS,
                               "peak_source": PEAK_SOURCE + " (FP32)"},
        "rel_err_hpsi_vs_oracle": eh, "rel_err_energies_vs_oracle": ee,
        "error_sample": "the first orbital of each cell against the FP64 oracle",
    }
    del psi, hp, rho, Vd
    torch.cuda.empty_cache()

    # ---- one orbital on a coarse 32^3 cell (fine 64^3), FP64: the single
    # call and a graph-captured plan (launch-bound at this size)
    n0 = (32, 32, 32)
    g0 = W.Grid(n0)
    p0 = torch.from_numpy(inputs.orbital(0, 0, n0)).to(dev)
    V0 = torch.from_numpy(inputs.gaussian_potential(0, 0, n0)).to(dev)
    o0 = torch.full((1,), 2.0, dtype=torch.float64, device=dev)
    r0 = torch.zeros(g0.fine, dtype=torch.float64, device=dev)
    ms_single = _time_steps(torch, lambda: W.hpsi_local(p0, V0, o0, g0, rho=r0), 20, 5)
    plan0 = W.Plan([g0], [0], prec=W.WVL_F64, graph=True)
    h0 = torch.empty_like(p0)
    e0k = torch.empty(1, dtype=torch.float64, device=dev)
    e0p = torch.empty_like(e0k)
    ms_plan = _time_steps(torch, lambda: plan0.hpsi(p0, [V0], o0, hpsi=h0, rho=[r0], ekin=e0k,
                                                    epot=e0p), 20, 5)
    out["config0_single_orbital"] = {
        "workload": "one orbital, periodic coarse 32^3 (fine 64^3), FP64, H psi + density + "
                    "energies",
        "ms_single_call": ms_single, "ms_graph_plan": ms_plan,
        "value": 1.0 / (ms_plan * 1e-3), "unit": UNIT,
        "checked": "tests/test_gpu_parity.py::test_config0_full (1e-12 against the oracle)",
    }
    del plan0

    # ---- single-pass FP64 sweep (one orbital, fine 32^3 .. 256^3): each 3D
    # operator is three 1D passes; per pass 16 compulsory bytes per point
    # (read + write) and 2 x taps flops per point
    sweep = {}
    gen = torch.Generator(device=dev)
    for nf in (32, 64, 128, 192, 256):
        gs = W.Grid((nf // 2,) * 3)
        pts = nf ** 3
        gen.manual_seed(9041543 + 1000 + nf)
        xs = (torch.rand((1, nf, nf, nf), generator=gen, dtype=torch.float64, device=dev) * 2 - 1)
        cs = xs.reshape(1, -1).clone()
        res_n = {}
        for name, taps, fn in (("magicfilter", 16, lambda: W.magicfilter(xs, gs)),
                               ("magicfilter_T", 16, lambda: W.magicfilter_T(xs, gs)),
                               ("kinetic", KIN_TAPS_ALGORITHMIC, lambda: W.kinetic(xs, gs)),
                               ("synthesis", 16, lambda: W.synthesis(cs, gs)),
                               ("analysis", 16, lambda: W.analysis(xs, gs))):
            ms_op = _time_steps(torch, fn, 5, 3)
            ms_pass = ms_op / 3
            t_roof = max(16.0 * pts / (HBM_GBS * 1e9), 2.0 * taps * pts / (FP64_PEAK_TFLOPS * 1e12))
            res_n[name] = {"ms_per_3d_operator": ms_op, "ms_per_pass": ms_pass,
                           "gb_per_s_per_pass": 16.0 * pts / (ms_pass * 1e-3) / 1e9,
                           "fp64_gflop_per_s": 2.0 * taps * pts / (ms_pass * 1e-3) / 1e9,
                           "roofline_frac": t_roof * 1e3 / ms_pass}
        sweep[f"{nf}^3"] = res_n
        del xs, cs
    out["pass_sweep_fp64"] = {
        "workload": "single 3D operators (three FP64 1D passes each) on one orbital, periodic, "
                    "fine 32^3, 64^3, 128^3, 192^3, 256^3, uniform[-1, 1] inputs from seed; "
                    "32^3 and 64^3 fit in L2",
        "roofline": "fraction of max(16 B per point / measured HBM bandwidth, 2 x taps flops "
                    "per point / FP64 peak measured by the FMA-chain probe in this run) per "
                    "pass (taps: 16, kinetic 29); every pass is FP64-pipe bound",
        "results": sweep,
    }
    torch.cuda.empty_cache()

    # ---- autograd, coarse 64^3 x 512 orbitals, FP32 forward + backward
    n = (64, 64, 64)
    g = W.Grid(n)
    norb = 512
    p = inputs.orbitals_device(4, norb, n, dev, torch.float32).requires_grad_(True)
    v = torch.from_numpy(inputs.gaussian_potential(4, 0, n)).to(dev).float().requires_grad_(True)
    occ = torch.full((norb,), 2.0, dtype=torch.float64, device=dev)

    def fwd_bwd():
        p.grad = None
        v.grad = None
        E = W.ELoc.apply(p, v, occ, g)
        E.backward()

    ms = _time_steps(torch, fwd_bwd, max(2, args.steps // 3), 2)
    out["autograd_fp32"] = {
        "workload": "E_loc(psi, V) forward + backward through ELoc, 512 orbitals, periodic "
                    "coarse 64^3 (fine 128^3), FP32 convolutions; backward recomputes "
                    "real-space psi and applies the adjoint chain",
        "value": norb / (ms * 1e-3), "unit": "orbital forward+backward/s", "ms_per_step": ms,
        "checked": "tests/test_gpu_autograd.py: FP64 central differences and oracle adjoint "
                   "on 4 orbitals at coarse 16^3",
    }
    del p, v
    torch.cuda.empty_cache()
    return out


def _run_ours(args, W, torch, dist, rank, world, local, dev):

    def barrier():
        if world > 1:
            dist.barrier()

    cell_of_orb, psi_h, Vs_h, occ_h = make_inputs(rank, args.per_cell)
    WL = workload(args.per_cell)
    cells = [W.Grid(s) for s in SIZES]
    f32 = args.prec == "f32"     # FP32 form of the same workload (profiling)
    emu = args.prec == "f64emu"  # FP64-accurate tensor-core form (profiling)
    if f32 or emu:
        WL["workload"] = WL["workload"].replace(
            "batched FP64", "batched FP32 convolutions (FP64 reductions)" if f32
            else "batched FP64 by f16-digit tensor-core emulation")
    pcode = W.WVL_F32 if f32 else (W.WVL_F64_EMU if emu else W.WVL_F64)
    tdt = torch.float32 if f32 else torch.float64
    if f32:
        psi_h = psi_h.astype(np.float32)
        Vs_h = [v.astype(np.float32) for v in Vs_h]
    chain = None if args.chain == "auto" else args.chain
    plan = W.Plan(cells, cell_of_orb, prec=pcode, graph=True,
                  autotune=not args.no_autotune, chain=chain)
    psi = torch.from_numpy(psi_h).to(dev)
    V = [torch.from_numpy(v).to(dev) for v in Vs_h]
    occ = torch.from_numpy(occ_h).to(dev)
    hp = torch.empty_like(psi)
    ek = torch.empty(len(cell_of_orb), dtype=torch.float64, device=dev)
    ep = torch.empty_like(ek)
    rho = [torch.zeros(c.fine, dtype=torch.float64, device=dev) for c in cells]
    if not args.no_autotune:
        plan.autotune(psi, V, occ, hpsi=hp, rho=rho)
    stream = torch.cuda.current_stream(dev)
    # several ranks: each holds its own orbitals of the same cells; a step
    # ends with the density and energy sums over the ranks
    en_sum = torch.zeros(2, dtype=torch.float64, device=dev)

    def step():
        if world > 1:
            for r in rho:
                r.zero_()
        plan.hpsi(psi, V, occ, hpsi=hp, rho=rho, ekin=ek, epot=ep)
        if world > 1:
            torch.stack([ek.sum(), ep.sum()], out=en_sum)
            sum_over_ranks(rho + [en_sum], dist, world)

    # ---- device-resident timed region (graph replay)
    gpu_id = local
    try:
        props = torch.cuda.get_device_properties(dev)
        gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else local
    except Exception:
        pass
    lp0 = W.kernel_launches()
    peaks = measure_pipe_peaks(W, gpu_id)
    probe_launches = W.kernel_launches() - lp0
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(gpu_id)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    l0 = W.kernel_launches()
    print(f"[bench] kernels enqueued before the timed region: {l0} "
          f"({l0 - probe_launches} without the pipe-peak probe)", file=sys.stderr, flush=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = W.kernel_launches() - l0

    # ---- per-stage times of the same steps, traced on the launching stream
    plan.set_profiling(True)
    plan.profile()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = plan.profile()
    plan.set_profiling(False)
    clk = clocks.stop()

    # ---- end to end through the public API from pinned host memory
    psi_pin = torch.from_numpy(psi_h).pin_memory()
    V_pin = [torch.from_numpy(v).pin_memory() for v in Vs_h]
    occ_pin = torch.from_numpy(occ_h).pin_memory()
    hp_pin = torch.empty(psi_h.shape, dtype=tdt).pin_memory()
    # the per-orbital energies travel in one 1 MiB buffer: on this system
    # device-to-host copies of a few KB block the host until the stream
    # drains, which would serialise the pipeline below
    nen = max(2 * len(cell_of_orb), 1 << 17)
    en_pin = torch.empty(nen, dtype=torch.float64).pin_memory()
    rho_pin = [torch.empty(c.fine, dtype=torch.float64).pin_memory() for c in cells]
    es = psi_pin.element_size()
    h2d = psi_pin.numel() * es + sum(v.numel() * es for v in V_pin) + occ_pin.numel() * 8
    d2h = hp_pin.numel() * es + en_pin.numel() * 8 + sum(r.numel() * 8 for r in rho_pin)

    # Pipelined steps: copies in on one stream, the plan on the compute
    # stream, copies out on a third; three device buffer sets (each with its
    # own plan and captured graph) let step k+1's inputs come in while step
    # k computes and step k-1's results go out, so the two copy directions
    # also overlap each other.  Every step still moves all of its inputs in
    # and all of its results out.
    ms_e2e = float("nan")
    e2e_ok = None
    if not args.no_e2e:
        comp = stream
        s_in = torch.cuda.Stream(dev)
        s_out = torch.cuda.Stream(dev)
        sets = []
        NSETS = 3
        for k in range(NSETS):
            if k == 0:
                bp, bpsi, bhp, brho, bV, bocc = plan, psi, hp, rho, V, occ
            else:
                bp = W.Plan(cells, cell_of_orb, prec=pcode,
                            graph=True, autotune=not args.no_autotune, chain=chain)
                bpsi, bhp = torch.empty_like(psi), torch.empty_like(hp)
                brho = [torch.empty_like(r) for r in rho]
                bV = [torch.empty_like(v) for v in V]
                bocc = torch.empty_like(occ)
                if not args.no_autotune:
                    bp.autotune(psi, V, occ, hpsi=bhp, rho=brho)
            ben = torch.zeros(nen, dtype=torch.float64, device=dev)
            no = len(cell_of_orb)
            sets.append(dict(plan=bp, psi=bpsi, hp=bhp, en=ben, ek=ben[:no], ep=ben[no:2 * no],
                             rho=brho, V=bV, occ=bocc,
                             ev_in=torch.cuda.Event(), ev_comp=torch.cuda.Event(),
                             ev_out=torch.cuda.Event()))
        for b in sets:
            b["ev_out"].record(s_out)

        def e2e_step(k):
            b = sets[k % NSETS]
            s_in.wait_event(b["ev_out"])           # the set's previous results are out
            with torch.cuda.stream(s_in):
                b["psi"].copy_(psi_pin, non_blocking=True)
                for v, vp in zip(b["V"], V_pin):
                    v.copy_(vp, non_blocking=True)
                b["occ"].copy_(occ_pin, non_blocking=True)
            b["ev_in"].record(s_in)
            comp.wait_event(b["ev_in"])
            for r in b["rho"]:
                r.zero_()
            b["plan"].hpsi(b["psi"], b["V"], b["occ"], hpsi=b["hp"], rho=b["rho"],
                           ekin=b["ek"], epot=b["ep"])
            sum_over_ranks(b["rho"], dist, world)
            b["ev_comp"].record(comp)
            s_out.wait_event(b["ev_comp"])
            with torch.cuda.stream(s_out):
                hp_pin.copy_(b["hp"], non_blocking=True)
                en_pin.copy_(b["en"], non_blocking=True)
                for r, rp in zip(b["rho"], rho_pin):
                    rp.copy_(r, non_blocking=True)
            b["ev_out"].record(s_out)

        for k in range(max(NSETS, args.warmup)):
            e2e_step(k)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e0.record(s_in)
        for k in range(args.steps):
            e2e_step(k)
        e1.record(s_out)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t0))
        # every step had the same inputs: the host copy of the last step's
        # H psi must equal the device-resident result bit for bit
        e2e_ok = bool(torch.equal(hp_pin, hp.cpu()))

    ms, ms_e2e = max_over_ranks([ms, ms_e2e], dist, world, dev)
    value = job_throughput(len(cell_of_orb), world, args.steps, ms)
    value_e2e = job_throughput(len(cell_of_orb), world, args.steps, ms_e2e)

    # roofline of the dominant kernel (kinetic pass, 3 launches per step)
    kin_ms, kin_launches = prof["kinetic"]
    pts = WL["fine_points_per_step"]
    flops_per_launch = 2.0 * KIN_TAPS_ALGORITHMIC * pts
    kin_avg_s = kin_ms * 1e-3 / max(kin_launches * 3, 1)
    achieved = flops_per_launch / kin_avg_s / 1e12 if kin_launches else None
    achieved_applied = (2.0 * KIN_TAPS_APPLIED * pts / kin_avg_s / 1e12) if kin_launches else None
    # DRAM bytes of one kinetic pass-1 launch from an ncu capture of the small
    # profiling case (36 orbitals, 33.6 M fine points, --per-cell 12), scaled
    # to this launch by the fine points processed; null for any other workload.
    traffic = (1029.2e6 * pts / 33619968) if (args.per_cell == PER_CELL and args.prec == "f64") else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                "traffic": traffic, "kernel": "kinetic 1D pass (FP64 DFMA pipe)",
                "flops_per_point": 2 * KIN_TAPS_ALGORITHMIC,
                "achieved_applied_taps": achieved_applied,
                "frac_applied_taps": (achieved_applied / FP64_PEAK_TFLOPS) if achieved else None,
                "frac_of_nominal": (achieved / FP64_PEAK_NOMINAL) if achieved else None,
                "peak_source": PEAK_SOURCE + " (FP64); nominal 1.25 TFLOP/s"}
    if emu:
        roofline["kernel"] = ("kinetic 1D pass, tensor-core emulation: FP64-equivalent rate "
                              "against the FP64 pipe's peak (the kernel itself is latency-bound "
                              "around its tensor-core MMAs)")
    chain_line = [ln for ln in plan.describe().splitlines() if ln.startswith("chain:")][0][7:]
    if f32:
        # FP32 form: the whole step against the slower of its HBM bytes and its
        # FP32 FMAs (the chain's kernels do not split into one dominant kernel)
        bpp = FUSED_BPP if chain_line.startswith("fused") else PASSES_BPP
        s_step = ms / args.steps * 1e-3
        gbs = bpp * pts / s_step / 1e9
        tfs = 2 * FP32_FMA_PER_POINT * pts / s_step / 1e12
        if bpp * pts / (HBM_GBS * 1e9) >= 2 * FP32_FMA_PER_POINT * pts / (FP32_PEAK_TFLOPS * 1e12):
            roofline = {"bound": "hbm", "achieved": gbs, "peak": HBM_GBS, "unit": "GB/s",
                        "frac": gbs / HBM_GBS, "traffic": None,
                        "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"}
        else:
            roofline = {"bound": "alu", "achieved": tfs, "peak": FP32_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": tfs / FP32_PEAK_TFLOPS, "traffic": None,
                        "peak_source": PEAK_SOURCE + " (FP32)"}
        roofline["kernel"] = (f"whole FP32 step ({chain_line}): {bpp:.0f} B and "
                              f"{FP32_FMA_PER_POINT:.0f} FMAs per orbital point")

    line = {
        "metric": (METRIC.replace("(FP64,", "(FP32 convolutions,") if f32 else
                   METRIC.replace("(FP64,", "(FP64 by f16-digit tensor-core emulation,") if emu
                   else METRIC),
        "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if f32 else ("f64 (f16-digit tensor-core emulation)" if emu else "f64"),
        "data": "synthetic", "config": WL,
        "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "pipelined": "copies in / plan / copies out on "
                "three streams, three device buffer sets",
                "host_result_matches_device": e2e_ok},
        "gpu_launches": int(launches),
        **({"e2e": None} if args.no_e2e else {}),
        "roofline": roofline,
        "clocks": clk,
        "pipe_peaks": peaks,
        "stage_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in prof.items()},
        "chain": chain_line,
    }
    if rank == 0 and world == 1 and not args.no_variants and args.prec == "f64":
        line["variants"] = measure_variants(args, W, torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        off = offsets_of(cell_of_orb)
        done, secs = 0, 0.0
        while secs < 10.0:
            d, s = oracle_sample(cell_of_orb, psi_h, Vs_h, occ_h, off)
            done += d
            secs += s
        line["cpu_baseline"] = {
            "value": done / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} orbitals (one of each cell per round), FP64 numpy oracle, "
                      f"single thread, {secs:.1f} s"}
        par, nw, ndone = oracle_all_cores()
        line["cpu_baseline_all_cores"] = {
            "value": par, "unit": UNIT, "cores": nw, "kind": "oracle",
            "sample": f"{ndone} orbitals over the three cells, one single-threaded oracle "
                      f"process per core ({nw}), value = cores / mean seconds per orbital"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-cell", type=int, default=PER_CELL,
                    help="orbitals per cell (64 = the benchmark workload; smaller for ncu)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--prec", choices=["f64", "f32", "f64emu"], default="f64",
                    help="f32 / f64emu run the FP32 / tensor-core FP64 form of the same "
                         "workload (profiling)")
    ap.add_argument("--chain", choices=["auto", "fused", "passes"], default="auto",
                    help="kernels of the local Hamiltonian: the autotuner's choice, the fused "
                         "plane/column kernels, or the transposing 1D passes")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP32 and autograd forms reported beside the FP64 line")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
