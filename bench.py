#!/usr/bin/env python
"""Benchmark of the GB300 core-excitation BSE hot path.

One step = one Haydock iteration (Sec. 3.2, Eq. 9) on the L2,3-edge workload
with multiplets (6 core states, 8^3 k-points, 64 bands, 16^3 grid, 36
local-basis functions): one application of H (band->grid, k->R x W R->k,
grid->band, diagonal, spin-orbit, short range) plus the FP64 recursion.
The metric is H psi matvecs per second.  Inputs are resident in HBM before
the timed region; u_nk alone is 1.07 GB (complex64-equivalent) > L2, so no
L2 flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W] [--precision split_bf16|fp32|fp64]
  python bench.py --impl reference     # the FP64 CPU oracle on this host's cores

Under torchrun each rank runs an independent replica on its own GPU
("replicas only": the path has no data exchange); value = all ranks' matvecs
/ the slowest rank's time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BSE H·ψ matvecs/s and GMRES solves/s at spectrum err ≤1e-4 vs FP64 plain"
WORKLOAD = "l23_multiplet"
WORKLOAD_DESC = ("L2,3 edge with multiplets: 6 core states (SO split 5.7 eV), k-mesh 8x8x8, Nb=64, "
                 "grid 16^3, W=-erf(r/0.5)/(5r), 36 local-basis functions, random Hermitian M (0.5 eV)")


def workload_desc(name):
    """Human-readable description of a workload (the generator's sizes when it is not the default one)."""
    if name == WORKLOAD:
        return WORKLOAD_DESC
    from paper_1601_07728_gb300 import synth as S
    c = S.CONFIGS.get(name, {})
    return "%s: %s" % (name, ", ".join("%s=%s" % kv for kv in sorted(c.items()))) if c else name


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default=os.environ.get("BSE_BENCH_PRECISION", "split_bf16"))
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--cpu-seconds", type=float, default=20.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tiles", default="auto",
                   help="tensor-core tiles of the headline run: auto (timed search) or SPLIT_K,STAGES[,SLABS]")
    p.add_argument("--polarisations", type=int, default=3,
                   help="start vectors of the batched-polarisation Haydock measurement (<= 1: skip)")
    p.add_argument("--gmres-omega", type=int, default=200, help="shifts in the GMRES measurement (0 = skip)")
    p.add_argument("--gmres-max-iter", type=int, default=2000)
    p.add_argument("--gmres-chunk", type=int, default=200, help="systems per batched H application")
    p.add_argument("--gmres-jacobi-omega", type=int, default=40,
                   help="shifts (every n-th of the GMRES set) of the Jacobi-preconditioned comparison")
    p.add_argument("--gmres-fp64-omega", type=int, default=4,
                   help="shifts (every n-th of the GMRES set) also solved by the plain FP64 form (0 = skip)")
    p.add_argument("--train-omega", type=int, default=16, help="training shifts of the learned preconditioner")
    p.add_argument("--train-epochs", type=int, default=10)
    p.add_argument("--train-systems", type=int, default=2,
                   help="seeded variants of the workload the preconditioner is trained on (0: the measured system)")
    p.add_argument("--apply-only", action="store_true",
                   help="time --steps applications of H to --apply-vectors vectors at once and exit")
    p.add_argument("--apply-vectors", type=int, default=200)
    p.add_argument("--fp64-steps", type=int, default=10,
                   help="captured Haydock steps of the plain FP64 form on the same workload (0 = skip)")
    p.add_argument("--supercell-steps", type=int, default=20,
                   help="timed Haydock steps on the 48^3-grid supercell workload (0 = skip)")
    p.add_argument("--no-one-pass", action="store_true",
                   help="skip the leg that times the one-pass schedule (bse_set_schedule one_pass)")
    p.add_argument("--one-pass-lag", type=int, default=2,
                   help="one-pass schedule: slabs read once but not yet twice, beyond the current one")
    p.add_argument("--sites", type=int, default=8,
                   help="sites of the many-site workload run in one batched launch of 200 steps (0 = skip)")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x, dist, device="cuda"):
    """The slowest rank's value of a per-rank time (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds_max, world):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            bid = f[0].lower()
            if self.bus_id and not (bid.endswith(self.bus_id[-12:]) or self.bus_id.endswith(bid[-12:])):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel class (one H psi, nc columns)
# ---------------------------------------------------------------------------
def algorithmic_bytes(s, prec, n_vec=1):
    nk, nx, nb, na, npj = s.n_k, s.n_x, s.n_bands, s.n_alpha, s.n_proj
    nc = na * n_vec
    u_elem = {"fp64": 16, "fp32": 8, "split_bf16": 8}[prec]     # bytes per complex u_nk(x)
    phi_elem = 16 if prec == "fp64" else 8
    vec = nc * nk * nb * 16
    u = nk * nx * nb * u_elem
    phi = nk * nx * nc * phi_elem
    w = nk * nx * (8 if prec == "fp64" else 4)
    out = {
        "band_to_grid": u + vec + phi,
        "kconv": 2 * phi + w,
        "grid_to_band": u + phi + 2 * vec + npj * nk * nb * 16 + nk * nb * 8,
    }
    if prec == "split_bf16":
        # bf16 hi+lo copies of phi' written by the k-conv and read by grid->band
        out["kconv"] = phi + nk * nx * nc * 8 + w
        out["grid_to_band"] = u + nk * nx * nc * 8 + 2 * vec + npj * nk * nb * 16 + nk * nb * 8
    return out


def u_bytes(s, prec="split_bf16"):
    """Bytes of one streamed copy of u_nk (complex64-equivalent for the reduced forms)."""
    return s.n_k * s.n_x * s.n_bands * (16 if prec == "fp64" else 8)


def matvec_flops(s):
    """Real flops of the two band<->grid contractions of one H psi (8 per complex MAC each)."""
    return 2 * 8 * s.n_k * s.n_x * s.n_bands * s.n_alpha


def timed_haydock(sysg, db, steps, stream, warmup=2):
    """Device time (ms) of one captured Haydock run of `steps` steps after a short warm-up."""
    import torch
    nv = 1 if db.ndim == 1 else db.shape[0]
    a = torch.zeros((nv, steps), dtype=torch.float64, device="cuda")
    bb = torch.zeros((nv, steps + 1), dtype=torch.float64, device="cuda")
    st = torch.zeros(nv, dtype=torch.int32, device="cuda")
    w = max(1, warmup)
    sysg.haydock(db, w, a=a[:, :w].contiguous(), bcoef=bb[:, :w + 1].contiguous(), steps=st)
    sysg.haydock(db, steps, a=a, bcoef=bb, steps=st)   # builds the graph the timed call relaunches
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sysg.haydock(db, steps, a=a, bcoef=bb, steps=st)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), int(st.sum().item()), a, bb, st


def cpu_oracle_rate(s, b, seconds, max_steps=None):
    """Haydock steps of the FP64 oracle on this host (untuned), bounded by time."""
    from oracle import bse_oracle as O
    import numpy as np
    v = b / np.linalg.norm(b)
    vp = np.zeros_like(v)
    bprev = 0.0
    n = 0
    t0 = time.perf_counter()
    while True:
        w = O.apply_h(s, v)
        a = float(np.real(np.vdot(v, w)))
        w = w - a * v - bprev * vp
        bn = float(np.linalg.norm(w))
        vp, v, bprev = v, w / bn, bn
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_steps and n >= max_steps):
            return n, el


def oracle_rate_one_thread(workload, steps=3):
    """The oracle on one host thread: this script's reference arm in a child
    process with every BLAS / OpenMP pool pinned to one thread."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env.pop("RANK", None)
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--workload", workload,
                            "--steps", str(steps), "--warmup", "1"], env=env, capture_output=True, text=True,
                           timeout=600)
        line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
        return float(json.loads(line)["value"])
    except Exception:
        return None


def reference_arm(args):
    import numpy as np
    from paper_1601_07728_gb300 import synth as S
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s = S.make_system(args.workload)
    b = S.make_start_vectors(s, 1)[0]
    cpu_oracle_rate(s, b, 0.0, max_steps=max(1, min(args.warmup, 2)))
    budget = 90.0
    n, el = cpu_oracle_rate(s, b, budget, max_steps=args.steps)
    rate = n / el
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "matvecs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / rate, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": workload_desc(args.workload), "precision": "fp64 (NumPy/SciPy oracle)"},
        "cpu_baseline": {"value": rate, "unit": "matvecs/s", "cores": cores, "kind": "oracle",
                         "sample": "%d FP64 oracle Haydock steps of the full workload (timed steps capped at "
                                   "%.0f s of CPU time)" % (n, budget)},
        "e2e": {"value": rate, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def apply_only(args, s, dist, world, rank):
    """H psi on --apply-vectors vectors in one pass (all columns of the
    tensor-core contractions at once), --steps timed applications after
    --warmup: matvecs/s and the FLOP rate of the two contractions."""
    import numpy as np
    import torch
    from paper_1601_07728_gb300 import bse, synth as S
    nv = args.apply_vectors
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    g = bse.System(s, precision=args.precision, max_vec=nv, stream=stream.cuda_stream)
    psi = torch.from_numpy(S.complex_normal(np.random.default_rng(0), (nv, s.dim))).to("cuda")
    out = torch.empty_like(psi)
    for _ in range(max(args.warmup, 1)):
        g.apply_h(psi, out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.apply_h(psi, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist)
    fl = 2 * 8.0 * s.n_k * s.n_x * s.n_bands * s.n_alpha * nv
    if rank == 0:
        print(json.dumps({"mode": "apply_only", "workload": args.workload, "precision": args.precision,
                          "vectors": nv, "columns": nv * s.n_alpha, "ms_per_application": ms,
                          "matvecs_per_s": job_rate(nv, ms / 1e3, world),
                          "contraction_tflops": fl / (ms / 1e3) / 1e12}), flush=True)
    g.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    from paper_1601_07728_gb300 import bse, synth as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    s = S.make_system(args.workload)
    b = S.make_start_vectors(s, 1)[0]
    if args.apply_only:
        return apply_only(args, s, dist, world, rank)
    # a dedicated (capturable) stream: the library records each Haydock run as one CUDA graph
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sysg = bse.System(s, precision=args.precision, max_vec=1, stream=stream.cuda_stream)
    if args.tiles == "auto":
        tiles = sysg.autotune(n_vec=1, reps=5)   # timed tile search (split-K, pipeline stages), before any timing
        tiles_by = "bse_autotune timed search"
    else:
        tiles = tuple(int(v) for v in args.tiles.split(","))
        sysg.set_tiles(*tiles[:2])
        if len(tiles) > 2:
            sysg.set_slabs(tiles[2])
        tiles_by = "fixed (--tiles)"
    n = sysg.dim
    db = torch.from_numpy(b).to("cuda")
    K, W = args.steps, args.warmup
    a_d = torch.zeros(K, dtype=torch.float64, device="cuda")
    b_d = torch.zeros(K + 1, dtype=torch.float64, device="cuda")
    st_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    # warm-up: W Haydock steps, then one untimed run of the timed call itself,
    # which builds the step-loop graph the library relaunches for a repeat of
    # the same call (graph instantiation is set-up, like bse_setup)
    sysg.haydock(db, max(W, 1), a=a_d[:max(W, 1)].contiguous(), bcoef=b_d[:max(W, 1) + 1].contiguous(),
                 steps=st_d)
    sysg.haydock(db, K, a=a_d, bcoef=b_d, steps=st_d)
    torch.cuda.synchronize()

    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        try:
            p = torch.cuda.get_device_properties(local)
            bus = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            bus = None
    clk = ClockSampler(str(bus) if bus else None)
    clk.start()
    time.sleep(0.5)
    l0 = sysg.launches
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sysg.haydock(db, K, a=a_d, bcoef=b_d, steps=st_d)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = sysg.launches - l0
    clocks = clk.stop()
    # per-kernel CUDA-event durations: the same Haydock run again with the
    # library's launch events on (recorded as event nodes of the captured step
    # graph, on the streams the kernels run on; the headline number above is
    # taken without them)
    kp = min(K, 100)
    ap = torch.zeros(kp, dtype=torch.float64, device="cuda")
    bp = torch.zeros(kp + 1, dtype=torch.float64, device="cuda")
    sysg.profile(True)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    sysg.haydock(db, kp, a=ap, bcoef=bp, steps=st_d)
    f1.record(stream)
    torch.cuda.synchronize()
    prof_ms_per_step = f0.elapsed_time(f1) / kp
    prof = sysg.profile_read()
    sysg.profile(False)
    sysg.haydock(db, K, a=a_d, bcoef=b_d, steps=st_d)   # restore the K-step result for steps_done
    t_max = max_over_ranks(ms, dist)
    steps_done = int(st_d.item())
    value = job_rate(steps_done, t_max / 1e3, world)

    # spectrum error against the FP64 oracle's stored 200-step Haydock run of
    # the same workload and start vector (tests/golden, written by the oracle
    # only): a separate 200-step run of this form, whatever --steps is, both
    # spectra evaluated by the same continued fraction on the 2000-point grid
    spec = None
    om = np.linspace(-5.0, 30.0, 2000)
    gold = os.path.join(ROOT, "tests", "golden", "%s_haydock200.npz" % args.workload)
    if os.path.exists(gold):
        g = np.load(gold)
        kk = int(g["steps"])
        a200, b200, st200 = sysg.haydock(b, kk)[:3]
        sg = bse.cf_spectrum(a200, b200, st200, om, 0.5)[0]
        so = bse.cf_spectrum(g["a"][:kk], g["b"][:kk + 1], kk, om, 0.5)[0]
        spec = {"steps": int(st200[0]), "rel_l2_vs_fp64_oracle": float(np.linalg.norm(sg - so) / np.linalg.norm(so)),
                "max_rel_vs_fp64_oracle": float(np.abs(sg - so).max() / np.abs(so).max()),
                "grid": "2000 omega in [-5, 30] eV, Gamma 0.5 eV",
                "reference": "stored FP64 oracle Haydock run (tests/golden/%s_haydock200.npz)" % args.workload}

    # the plain FP64 form on the same workload: a few captured steps
    fp64_form = None
    if args.fp64_steps > 0:
        sys64 = bse.System(s, precision="fp64", max_vec=1, stream=stream.cuda_stream)
        ms64, done64, _, _, _ = timed_haydock(sys64, db, args.fp64_steps, stream)
        sys64.close()
        ms64 = max_over_ranks(ms64, dist)
        fl = matvec_flops(s)
        fp64_form = {"matvecs_per_s": job_rate(done64, ms64 / 1e3, world), "ms_per_step": ms64 / args.fp64_steps,
                     "steps": args.fp64_steps, "gflop_per_matvec": fl / 1e9,
                     "tflops": fl * done64 / (ms64 / 1e3) / 1e12, "fp64_peak_tflops_nominal": 1.25,
                     "frac_of_nominal_fp64": fl * done64 / (ms64 / 1e3) / 1e12 / 1.25,
                     "speedup_of_headline": value / job_rate(done64, ms64 / 1e3, world)}

    # three polarisations (start vectors) advanced together: one pass over u_nk
    # per step serves all three H psi (GEMM columns 3 x 6); the first vector is
    # the headline's start vector, so its spectrum is checked against the same
    # stored oracle run
    pol = None
    if args.polarisations > 1:
        npol = args.polarisations
        sys3 = bse.System(s, precision=args.precision, max_vec=npol, stream=stream.cuda_stream)
        sys3.autotune(n_vec=npol, reps=5)
        b3 = torch.from_numpy(S.make_start_vectors(s, npol)).to("cuda")
        a3 = torch.zeros((npol, K), dtype=torch.float64, device="cuda")
        bb3 = torch.zeros((npol, K + 1), dtype=torch.float64, device="cuda")
        st3 = torch.zeros(npol, dtype=torch.int32, device="cuda")
        sys3.haydock(b3, max(W, 1), a=a3[:, :max(W, 1)].contiguous(), bcoef=bb3[:, :max(W, 1) + 1].contiguous(),
                     steps=st3)
        sys3.haydock(b3, K, a=a3, bcoef=bb3, steps=st3)   # builds the graph the timed call relaunches
        torch.cuda.synchronize()
        barrier()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        sys3.haydock(b3, K, a=a3, bcoef=bb3, steps=st3)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(p0.elapsed_time(p1), dist)
        done3 = int(st3.sum().item())
        pol = {"n_vec": npol, "matvecs_per_s": job_rate(done3, pms / 1e3, world), "ms_per_step": pms / K,
               "note": "polarisations batched as GEMM columns; u_nk read once per step for all of them"}
        if spec is not None:
            k3 = min(K, int(g["steps"]))
            s0 = bse.cf_spectrum(a3[0].cpu().numpy()[:k3], bb3[0].cpu().numpy()[:k3 + 1], k3, om, 0.5)[0]
            r0 = bse.cf_spectrum(g["a"][:k3], g["b"][:k3 + 1], k3, om, 0.5)[0]
            pol["spectrum_steps"] = k3
            pol["rel_l2_vs_fp64_oracle_vector0"] = float(np.linalg.norm(s0 - r0) / np.linalg.norm(r0))
        sys3.close()
        del b3

    # the one-pass schedule (one persistent kernel per H psi, u_nk streamed from
    # HBM once when the slabs between its two reads stay in L2): the headline's
    # workload, start vector and step count, timed the same way
    onep = None
    if not args.no_one_pass and args.precision == "split_bf16":
        sys1 = bse.System(s, precision=args.precision, max_vec=1, stream=stream.cuda_stream)
        try:
            sys1.set_schedule("one_pass", lag=args.one_pass_lag)
        except bse.BSEError as ex:
            onep = {"unavailable": str(ex)}
        else:
            ms1, done1, _, _, _ = timed_haydock(sys1, db, K, stream)
            ms1 = max_over_ranks(ms1, dist)
            sys1.profile(True)
            sys1.haydock(db, kp, a=ap, bcoef=bp, steps=st_d)
            torch.cuda.synchronize()
            n1, t1 = sys1.profile_read()["one_pass"]
            sys1.profile(False)
            ab = algorithmic_bytes(s, args.precision)
            u1 = u_bytes(s, args.precision)
            # one read of u_nk plus everything else the three two-pass kernels move
            alg1 = ab["band_to_grid"] + ab["kconv"] + ab["grid_to_band"] - u1
            k_ms = t1 / max(n1, 1)
            pk, _ = peaks()
            onep = {"matvecs_per_s": job_rate(done1, ms1 / 1e3, world), "ms_per_step": ms1 / K, "steps": K,
                    "lag": args.one_pass_lag, "stages": 5, "kernel_ms": k_ms, "kernel_launches": n1,
                    "alg_bytes_per_launch": alg1, "achieved_gbs": alg1 / (k_ms / 1e3) / 1e9,
                    "frac_of_hbm_peak": alg1 / (k_ms / 1e3) / 1e9 / pk,
                    "two_read_bytes_frac": (alg1 + u1) / (k_ms / 1e3) / 1e9 / pk,
                    "headline_over_one_pass": value / job_rate(done1, ms1 / 1e3, world),
                    "note": "frac_of_hbm_peak counts u_nk once; two_read_bytes_frac counts the bytes of the "
                            "two-pass step (u_nk twice), so it can exceed 1"}
            try:
                with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
                    onep["dram_bytes_per_launch"] = json.load(f).get("%s/%s/one_pass" % (args.workload,
                                                                                       args.precision))
            except Exception:
                pass
        sys1.close()

    # GMRES: (H - omega - i Gamma) x = b for n_omega shifts, all advanced together
    gm = None
    if args.gmres_omega > 0:
        n_om = args.gmres_omega
        zs = np.linspace(-5.0, 30.0, n_om) + 0.5j
        sys_g = bse.System(s, precision=args.precision, max_vec=args.gmres_chunk, stream=stream.cuda_stream)
        sys_g.autotune(n_vec=args.gmres_chunk, reps=3)
        xg = torch.empty((n_om, n), dtype=torch.complex128, device="cuda")
        sys_g.gmres(db, zs[:2], rtol=1e-3, restart=30, max_iter=60, precond="none", x=xg[:2])   # warm-up
        gm = {"n_omega": n_om, "rtol": 1e-6, "restart": 30, "max_iter": args.gmres_max_iter,
              "shifts": "omega in linspace(-5, 30, %d) eV + 0.5i" % n_om, "chunk": args.gmres_chunk}
        def leg(system, pc, z, x):
            torch.cuda.synchronize()
            barrier()
            l1 = system.launches
            g0 = time.perf_counter()
            _, g_it, g_rr, g_st = system.gmres(db, z, rtol=1e-6, restart=30, max_iter=args.gmres_max_iter,
                                               precond=pc, x=x)
            torch.cuda.synchronize()
            g_el = max_over_ranks(time.perf_counter() - g0, dist)
            conv = int(np.sum(g_rr <= 1e-6))
            return {"solves_per_s": job_rate(conv, g_el, world), "seconds": g_el, "converged": conv, "n_omega": len(z),
                    "iters_mean": float(np.mean(g_it)), "iters_max": int(np.max(g_it)),
                    "max_rel_resid": float(np.max(g_rr)), "gpu_launches": system.launches - l1}

        def sigma_of(x):
            # sigma(omega) = (1/pi) Im <b|x(z)>
            return (torch.imag(x @ db.conj()) / np.pi).cpu().numpy()

        gm["none"] = leg(sys_g, "none", zs, xg)
        sig_none = sigma_of(xg)
        # Jacobi on an evenly spaced subset (it converges slowly at interior shifts)
        selj = np.linspace(0, n_om - 1, min(args.gmres_jacobi_omega, n_om)).round().astype(int)
        gm["jacobi"] = leg(sys_g, "jacobi", zs[selj], xg[:len(selj)])
        gm["jacobi"]["omega_subset"] = "every %.1f-th shift of the set" % (n_om / max(len(selj), 1))
        # learned preconditioner: the network's prior (last layer zero: the damped
        # diagonal) and the network after training on the GPU at shifts between the
        # measured ones (residual probes of plain GMRES(30), 10-step minimal-residual loss)
        net = bse.MLP(S.mlp_init(0))
        bse.attach_mlp(sys_g, net)
        # network inference alone: features + three dense layers (FP16 weights,
        # FP32 accumulate) for every row at one shift, device output
        net.outputs(sys_g, 10.0, 0.5)          # grows the network's row buffers once
        sys_g.profile(True)
        for _ in range(5):
            net.outputs(sys_g, 10.0, 0.5)
        n_inf, t_inf = sys_g.profile_read()["prep"]   # the feature and three dense-layer kernels
        sys_g.profile(False)
        inf_ms = t_inf / 5
        inf_fl = 2.0 * n * (12 * 128 + 128 * 128 + 128 * 34)
        gm["mlp_inference"] = {"ms_per_shift": inf_ms, "kernel_launches": n_inf // 5, "rows": n,
                               "tflops": inf_fl / (inf_ms / 1e3) / 1e12,
                               "gflop_per_shift": inf_fl / 1e9,
                               "note": "features + 12-128-128-34 network for every row at one shift (SIMT, FP16 "
                                       "weights, FP32 accumulate); a 200-shift build is 200 of these"}
        gm["mlp_prior"] = leg(sys_g, "mlp", zs, xg)
        if args.train_omega > 0:
            step = (zs[1].real - zs[0].real) if n_om > 1 else 1.0
            zt = np.linspace(-5.0 + 0.5 * step, 30.0 - 0.5 * step, args.train_omega) + 0.5j
            # training systems: seeded variants of the workload (other u_nk, band
            # energies, projectors and couplings), never the measured system
            if args.train_systems > 0:
                tr_sys, tr_b = [], []
                for k in range(1, args.train_systems + 1):
                    sk = S.make_system_device(dict(S.CONFIGS[args.workload]), site=k, name=args.workload)
                    tr_sys.append(bse.System(sk, precision=args.precision, max_vec=min(args.gmres_chunk, 16),
                                             stream=stream.cuda_stream))
                    tr_b.append(S.make_start_vectors(sk, 1)[0])
                    del sk
                torch.cuda.empty_cache()
                trained_on = "seeded variants (sites 1..%d) of the workload; evaluated on the held-out site 0" % (
                    args.train_systems)
            else:
                tr_sys, tr_b = [sys_g], [b]
                trained_on = "the measured system itself"
            torch.cuda.synchronize()
            t_tr = time.perf_counter()
            hist = net.train(tr_sys, tr_b, zt, epochs=args.train_epochs, batch=1, lr=1e-3, seed=1, steps=10)
            torch.cuda.synchronize()
            t_tr = time.perf_counter() - t_tr
            for g_ in tr_sys:
                if g_ is not sys_g:
                    g_.close()
            del tr_sys
            gm["mlp_trained"] = leg(sys_g, "mlp", zs, xg)
            gm["mlp_trained"]["training"] = {
                "seconds": t_tr, "shifts": args.train_omega, "epochs": args.train_epochs,
                "systems": max(1, args.train_systems), "trained_on": trained_on,
                "loss_first_epoch": float(hist[0]), "loss_last_epoch": float(hist[-1]),
                "note": "training shifts are the midpoints between measured shifts; training timed separately"}
        # one restart cycle (30 iterations) of the trained-network solve with the
        # library's launch timing on: where GMRES time goes, and the FLOP rate of
        # the band->grid contraction at this column count (first cycle: every
        # shift active, so each H application covers min(chunk, n_omega) shifts)
        sys_g.profile(True)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        _, it_c, _, _ = sys_g.gmres(db, zs, rtol=1e-6, restart=30, max_iter=30, precond="mlp", x=xg)
        c1.record(stream)
        torch.cuda.synchronize()
        cyc_ms = c0.elapsed_time(c1)
        prof_g = sys_g.profile_read()
        sys_g.profile(False)
        n_apply = int(np.sum(it_c)) + n_om                   # Arnoldi applications + one true residual each
        fl = 8.0 * s.n_k * s.n_x * s.n_bands * s.n_alpha * n_apply   # real flops of one contraction over the cycle
        nb2g, tb2g = prof_g["band_to_grid"]
        peaks_d = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks_d = json.load(f)
        except Exception:
            pass
        bf16_sus = float(peaks_d.get("bf16_tflops_sustained", 1700.0))
        alg_tf = fl / (tb2g / 1e3) / 1e12 if tb2g > 0 else None
        gm["one_cycle_breakdown"] = {
            "ms": cyc_ms, "h_applications": n_apply, "columns_per_pass": min(args.gmres_chunk, n_om) * s.n_alpha,
            "kernels_ms": {k: round(v[1], 3) for k, v in prof_g.items() if v[0]},
            "band_to_grid_roofline": {
                "bound": "tensor", "unit": "TFLOP/s", "alg_tflops": alg_tf,
                "tensor_tflops": None if alg_tf is None else 3 * alg_tf,
                "peak": bf16_sus, "peak_kind": "measured bf16 sustained" if peaks_d else "fallback",
                "frac": None if alg_tf is None else 3 * alg_tf / bf16_sus, "launches": nb2g,
                "note": "split-bf16 runs three bf16 MMAs per product (hi*hi + hi*lo + lo*hi): tensor work "
                        "= 3 x the complex contraction's 8 real flops per MAC"}}
        bse.attach_mlp(sys_g, None)
        del net
        if args.gmres_fp64_omega > 0:
            # plain FP64 form on a subset of the shifts, and the spectrum difference
            # sigma = Im<b|x>/pi between this form and it at those shifts
            sel = np.linspace(0, n_om - 1, min(args.gmres_fp64_omega, n_om)).round().astype(int)
            sys64 = bse.System(s, precision="fp64", max_vec=len(sel), stream=stream.cuda_stream)
            x64 = torch.empty((len(sel), n), dtype=torch.complex128, device="cuda")
            gm["fp64_none"] = leg(sys64, "none", zs[sel], x64)
            s64 = sigma_of(x64)
            gm["fp64_none"]["omega"] = [float(v) for v in zs[sel].real]
            gm["sigma_rel_err_vs_fp64"] = float(np.linalg.norm(sig_none[sel] - s64) / np.linalg.norm(s64))
            sys64.close()
            del x64
        sys_g.close()
        del xg

    peak, peak_kind = peaks()

    # the 48^3-grid supercell workload (6 core states, 2^3 k, 1024 bands, 36
    # local functions; u_nk 14.5 GB complex128 drawn on the device): captured
    # Haydock steps of one start vector and of three polarisations batched
    sc = None
    if args.supercell_steps > 0:
        import torch as _t
        cfg4 = S.CONFIGS["supercell_48"]
        s4 = S.make_system_device(cfg4, name="supercell_48")
        b4 = S.make_start_vectors(s4, 3)
        sc = {"workload": "supercell_48", "desc": workload_desc("supercell_48"), "steps": args.supercell_steps}
        for nv in (1, 3):
            g4 = bse.System(s4, precision=args.precision, max_vec=nv, stream=stream.cuda_stream)
            tiles4 = g4.autotune(n_vec=nv, reps=3)
            db4 = _t.from_numpy(b4[:nv] if nv > 1 else b4[0]).to("cuda")
            ms4, done4, _, _, _ = timed_haydock(g4, db4, args.supercell_steps, stream)
            g4.close()
            ms4 = max_over_ranks(ms4, dist)
            per_step = ms4 / args.supercell_steps / 1e3
            ub = u_bytes(s4, args.precision)
            leg4 = {"matvecs_per_s": job_rate(done4, ms4 / 1e3, world), "ms_per_step": per_step * 1e3,
                    "spectra_per_s_300_steps": job_rate(nv, per_step * 300, world),
                    "tiles": {"grid_to_band_split_k": tiles4[0], "pipeline_stages": tiles4[1]},
                    "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": peak_kind,
                                 "alg_bytes_per_step": 2 * ub, "achieved": 2 * ub / per_step / 1e9,
                                 "frac": 2 * ub / per_step / 1e9 / peak,
                                 "note": "two streams of u_nk per step (band->grid, grid->band)"}}
            sc["n_vec_%d" % nv] = leg4
            del db4
        del s4
        _t.cuda.empty_cache()

    # many absorbing sites of uneven size (k mesh n^3, n = 4..8; grid m^3,
    # m = 12..20; 32..256 bands; 1 or 6 core states): the first --sites sites
    # of the seeded 64-site set, one graph-captured launch of 200 Haydock steps
    sites = None
    if args.sites > 0:
        import torch as _t
        n_s = args.sites
        systems, bsl, tot_u, tot_mv = [], [], 0, 0
        for i in range(n_s):
            cfg = S.batched_site_config(i)
            si = S.make_system_device(cfg, site=i, name="sites64")
            gi = bse.System(si, precision=args.precision, stream=_t.cuda.Stream().cuda_stream)
            gi.autotune(n_vec=1, reps=3)
            systems.append(gi)
            bsl.append(_t.from_numpy(S.make_start_vectors(si, 1, seed=i)).to("cuda"))
            tot_u += u_bytes(si, args.precision)
            del si
            _t.cuda.empty_cache()
        outs = [(_t.zeros((1, 200), dtype=_t.float64, device="cuda"), _t.zeros((1, 201), dtype=_t.float64, device="cuda"),
                 _t.zeros(1, dtype=_t.int32, device="cuda")) for _ in range(n_s)]
        bse.haydock_batch(systems, bsl, 3, outs=[(o[0][:, :3].contiguous(), o[1][:, :4].contiguous(), o[2])
                                                 for o in outs])   # warm-up
        _t.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        _, sts = bse.haydock_batch(systems, bsl, 200, outs=outs)
        _t.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, dist)
        done_s = int(sum(int(o[2].sum().item()) for o in outs))
        for gi in systems:
            gi.close()
        del systems, bsl, outs
        _t.cuda.empty_cache()
        sites = {"n_sites": n_s, "steps": 200, "seconds": el, "spectra_per_s": job_rate(n_s, el, world),
                 "matvecs_per_s": job_rate(done_s, el, world), "statuses_ok": bool(np.all(sts == 0)),
                 "u_bytes_total": tot_u,
                 "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": peak_kind,
                              "alg_bytes_per_batched_step": 2 * tot_u,
                              "achieved": 2 * tot_u * 200 / el / 1e9, "frac": 2 * tot_u * 200 / el / 1e9 / peak,
                              "note": "wall time of the one bse_haydock_batch call (graph capture and launch "
                                      "included); two streams of every site's u_nk per batched step"},
                 "sites": "batched_site_config(0..%d): uneven k meshes, grids, bands and core states" % (n_s - 1)}

    # end to end: the public call with pinned host buffers, H2D + D2H every step
    hp = torch.from_numpy(b).pin_memory()
    ho = torch.empty_like(hp).pin_memory()
    hpn, hon = hp.numpy(), ho.numpy()
    for _ in range(2):
        sysg.apply_h(hpn, hon)
    k_e2e = max(10, min(K, 100))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        sysg.apply_h(hpn, hon)
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, dist)
    e2e = job_rate(k_e2e, el, world)

    # roofline of the dominant kernel class
    dom = max(("band_to_grid", "kconv", "grid_to_band"), key=lambda k: prof[k][1])
    nl, tot = prof[dom]
    alg = algorithmic_bytes(s, args.precision)[dom]
    avg_s = tot / max(nl, 1) / 1e3
    achieved = alg / avg_s / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f)
        key = "%s/%s/%s" % (args.workload, args.precision, dom)
        traffic = tj.get(key)
    except Exception:
        pass

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            ns, el2 = cpu_oracle_rate(s, b, args.cpu_seconds)
            cpu = {"value": ns / el2, "unit": "matvecs/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "%d FP64 NumPy oracle Haydock steps of the same workload (%.1f s; BLAS-threaded "
                             "matmuls, single-threaded FFTs)" % (ns, el2)}
            # the same oracle on one thread, and on the 1s workload
            cpu["one_thread_matvecs_per_s"] = oracle_rate_one_thread(args.workload)
            s1 = S.make_system("k_edge_small")
            n1, e1 = cpu_oracle_rate(s1, S.make_start_vectors(s1, 1)[0], 2.0)
            cpu["k_edge_small_matvecs_per_s"] = n1 / e1
        dtype = {"fp64": "f64", "fp32": "f32", "split_bf16": "bf16x3"}[args.precision]
        line = {
            "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max / max(steps_done, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "desc": workload_desc(args.workload), "precision": args.precision,
                       "recursion": "f64 Haydock, no re-orthogonalisation", "n_vec": 1, "dim": n,
                       "l2": ("inputs larger than L2 (u_nk %.2f GB), no flush" % (u_bytes(s, args.precision) / 1e9)
                              if u_bytes(s, args.precision) > 129e6 else
                              "u_nk %.0f MB fits in L2: steps reuse it (a small case, not a headline)"
                              % (u_bytes(s, args.precision) / 1e6)),
                       "parallelism": "replicas",
                       "tiles": {"grid_to_band_split_k": tiles[0], "pipeline_stages": tiles[1],
                                 "x_slabs": sysg.slabs, "chosen_by": tiles_by}},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                         "alg_bytes_per_launch": alg, "avg_launch_ms": avg_s * 1e3, "launches": nl},
            "kernels_ms": {k: {"launches": v[0], "total_ms": round(v[1], 4)} for k, v in prof.items() if v[0]},
            "profiled_region": {"steps": kp, "ms_per_step": prof_ms_per_step},
            "e2e": {"value": e2e, "unit": "matvecs/s", "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": n * 16,
                    "api": "bse_apply_h with pinned host psi/hpsi"},
            "gpu_launches": launches,
            "spectrum": spec,
            "fp64_form": fp64_form,
            "polarisations": pol,
            "one_pass": onep,
            "supercell": sc,
            "sites": sites,
            "gmres": gm,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
