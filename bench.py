#!/usr/bin/env python
"""Throughput of the batched checkerboard Metropolis sweep on GB300.

Workload (synthetic, seeded): 512 Ising lattices with side L = 2^e, e uniform
in {5..11}, beta ~ U(0.3, 0.55), h ~ N(0, 0.05), J = 1, int8 spins, random
start; one step = one sweep (both checkerboard colours) of every lattice,
about 4.1e8 site updates.  The default run is the whole 2000-sweep job.  The
state (~409 MB, plus its ping-pong partner) is larger than the 129 MB L2, so
no flush is needed between steps.

One JSON line on stdout (rank 0):
  value        site-updates/s of the batched, graph-replayed launch form
  plain        the same workload in the plain per-lattice launch form
  roofline     the batched sweep kernel: algorithmic 2 B per site update
               (one int8 read, one write) / its CUDA-event launch time
  cpu_baseline the CPU oracle on this host's cores, a bounded sample
  e2e          end to end through the C ABI with host buffers: every step
               uploads the spins from pinned host memory (one bit per spin;
               int8 spins under e2e.int8_spins), sweeps, and reads back the
               spins and that step's statistics
--impl reference times the CPU oracle alone (the reference arm).
Multi-GPU (torchrun): the 512-lattice batch is split over the ranks by
site count (strong scaling: every lattice keeps the Philox stream it has in
the one-GPU run, no data-path collective); --scaling weak gives every rank the
whole batch under its own seed instead.  Time = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "site-updates/s and % HBM roofline, batched vs plain launch on 1 GB300 (bit-exact)"
UNIT = "site-updates/s"
WORKLOAD = ("uneven512: 512 Ising lattices, L=2^e with e uniform in {5..11}, beta~U(0.3,0.55), "
            "h~N(0,0.05), J=1, int8 spins, checkerboard Metropolis, one step = one sweep of all lattices")
SEED = 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=6)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=24)
    ap.add_argument("--cpu-sweeps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--scaling", default="strong", choices=["strong", "weak"],
                    help="N > 1: split one batch over the ranks (strong) or give each rank the whole batch (weak)")
    ap.add_argument("--workload", default="uneven512",
                    choices=["uneven512", "potts_q3", "potts_q8", "cpm1024", "ising_small", "few256", "grad", "mlp", "dmc",
                             "spinglass", "cpm_batch", "triangular", "nnn", "fit", "rng"])
    return ap.parse_args()


# ----------------------------------------------------------------- CPU oracle
def _oracle_lattice(args):
    import numpy as np

    import oracle
    i, d, seed, sweeps = args
    s = oracle.init_ising(d["L"], seed, i).copy()
    t0 = time.perf_counter()
    oracle.ising_run(s, d["beta"], d["J"], d["h"], seed, i, 0, sweeps, record=False)
    return d["L"] * d["L"] * sweeps, time.perf_counter() - t0


def cpu_oracle_rate(lats, sweeps, cores):
    """The oracle as it stands, one lattice per task on `cores` processes."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    tasks = [(i, d, SEED, sweeps) for i, d in enumerate(lats)]
    tasks.sort(key=lambda a: -a[1]["L"])
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_lattice, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    updates = sum(r[0] for r in res)
    return updates / wall, updates, wall


def _oracle_potts(args):
    import oracle
    i, d, seed, sweeps = args
    s = oracle.init_potts(d["L"], d["q"], seed, i).copy()
    t0 = time.perf_counter()
    oracle.potts_run(s, d["q"], d["beta"], d["J"], seed, i, 0, sweeps, record=False)
    return d["L"] * d["L"] * sweeps, time.perf_counter() - t0


DMC_SHAPE = (1024, 64, 1)   # lattices, side, relaxed sweeps per optimisation iteration


def dmc_targets(B, L):
    """Synthetic +-1 patterns: horizontal stripes, vertical stripes and blocks of
    widths 2..5 (the kind of target shown for the pattern optimisation)."""
    import numpy as np
    y = np.arange(L)[:, None] * np.ones((1, L))
    x = y.T
    out = np.empty((B, L, L), dtype=np.float32)
    for b in range(B):
        w = 2 + b % 4
        kind = (b // 4) % 3
        pat = (y // w) % 2 if kind == 0 else ((x // w) % 2 if kind == 1 else ((y // w + x // w) % 2))
        out[b] = np.where(pat == 0, 1.0, -1.0)
    return out


def _oracle_dmc(args):
    import numpy as np

    from oracle import dmc as odmc
    b0, n, L, K = args
    targets = dmc_targets(b0 + n, L)[b0:].astype(np.float64)
    t0 = time.perf_counter()
    for i in range(n):
        J = np.ones((2, L, L))
        s = np.ones((L, L))
        tape = odmc.run(s, J, 1 / 0.9, 0.0, 10.0, SEED, b0 + i, 0, K, tape=True)
        _, g = odmc.loss(s, targets[i])
        odmc.backward(tape, J, g, 1 / 0.9, 0.0, 10.0, SEED, b0 + i, 0)
    return n * L * L * K, time.perf_counter() - t0


def spinglass_couplings(B, L, seed=8):
    import numpy as np
    return np.random.default_rng(seed).choice([-1.0, 1.0], size=(B, 2, L, L)).astype(np.float32)


def _oracle_spinglass(args):
    import numpy as np

    from oracle import dmc as odmc
    b0, n = args
    L = 64
    J = spinglass_couplings(b0 + n, L)[b0:].astype(np.float64)
    rng = np.random.default_rng(b0)
    t0 = time.perf_counter()
    for i in range(n):
        s = rng.choice([-1.0, 1.0], size=(L, L))
        relaxed = s.copy()
        tape = odmc.run(relaxed, J[i], 2.0, 0.0, 10.0, SEED, b0 + i, 0, 1, tape=True)
        _, gE = odmc.energy(relaxed, J[i], 0.0)
        gs, _ = odmc.backward(tape, J[i], gE, 2.0, 0.0, 10.0, SEED, b0 + i, 0)
        odmc.discretize(odmc.spin_step(s, gs, 2.0))
    return n * L * L, time.perf_counter() - t0


def _oracle_cpm_batch(args):
    import oracle
    from paper_2304_01772_gb300 import workloads as wl
    b0, n = args
    p = wl.cpm_paper()
    op = oracle.CPM(L=p["L"], J=p["J"], lam=p["lam"], target=p["target"], n_cells=p["n_cells"], T=p["T"],
                    side=p["side"], cols=p["cols"])
    t0 = time.perf_counter()
    for b in range(b0, b0 + n):
        ids, types, vol = op.init(SEED, b)
        ids = ids.copy()
        op.run(ids, vol, types, SEED, b, 0, 2, record=False)
    return n * 2 * p["L"] ** 2, time.perf_counter() - t0


def _oracle_fit_chain(i):
    import oracle
    s = oracle.init_ising(256, SEED, i).copy()
    t0 = time.perf_counter()
    oracle.ising_run(s, 0.45, 1.0, 0.0, SEED, i, 0, 100)
    return 256 * 256 * 100, time.perf_counter() - t0


def _oracle_tri(args):
    import oracle
    b0, n = args
    t0 = time.perf_counter()
    for b in range(b0, b0 + n):
        s = oracle.init_ising(192, SEED, b).copy()
        oracle.tri_run(s, 0.2 + 0.15 * b / 255, 1.0, 0.0, SEED, b, 0, 1, record=False)
    return n * 192 * 192, time.perf_counter() - t0


def _oracle_nnn(args):
    import oracle
    from paper_2304_01772_gb300 import workloads as wl
    b0, n = args
    lats = wl.nnn256()
    t0 = time.perf_counter()
    for b in range(b0, b0 + n):
        d = lats[b]
        s = oracle.init_ising(d["L"], SEED, b).copy()
        oracle.nnn_run(s, d["beta"], d["J"], d["J2"], d["h"], SEED, b, 0, 1, record=False)
    return n * 256 * 256, time.perf_counter() - t0


def _oracle_rng(args):
    import oracle
    g0, n = args
    t0 = time.perf_counter()
    oracle.philox_xor(SEED, 0, 0, 0, g0, n)
    return 4 * n, time.perf_counter() - t0


def cpu_oracle_pool(fn, tasks, cores):
    import multiprocessing as mp

    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(fn, tasks, chunksize=1)
    wall = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    return units / wall, units, wall


def few256():
    """16 Ising lattices 256^2 across the critical point: a batch of fewer
    lattices than SMs (the resident form can split each over a cluster)."""
    return [dict(L=256, beta=0.3 + 0.25 * k / 15, J=1.0, h=0.0) for k in range(16)]


def cpu_baseline_secondary(workload, cores):
    """The oracle on a bounded sample of a secondary workload (before any GPU call)."""
    import numpy as np

    import oracle
    from paper_2304_01772_gb300 import workloads as wl
    if workload.startswith("potts"):
        q = int(workload[-1])
        lats = wl.potts_batch(q)
        pick = list(range(0, 64, 64 // cores))[:cores]
        rate, units, wall = cpu_oracle_pool(_oracle_potts, [(i, lats[i], SEED, 1) for i in pick], cores)
        return {"value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{len(pick)} of the 64 lattices, one sweep each ({wall:.1f} s wall)"}
    if workload == "rng":
        n = 1 << 25
        rate, units, wall = cpu_oracle_pool(_oracle_rng, [(i * n, n) for i in range(cores)], cores)
        return {"value": rate, "unit": "draws/s", "cores": cores, "kind": "oracle",
                "sample": f"{cores} x 2^25 Philox4x32-10 blocks, one range per core ({wall:.1f} s wall)"}
    if workload == "cpm1024":
        p = wl.cpm1024()
        op = oracle.CPM(L=p["L"], J=p["J"], lam=p["lam"], target=p["target"], n_cells=p["n_cells"], T=p["T"],
                        side=p["side"], cols=p["cols"])
        ids, types, vol = op.init(SEED, 0)
        ids = ids.copy()
        t0 = time.perf_counter()
        op.run(ids, vol, types, SEED, 0, 0, 2, record=False)
        wall = time.perf_counter() - t0
        return {"value": 2 * p["L"] ** 2 / wall, "unit": "copy-attempts/s", "cores": 1, "kind": "oracle",
                "sample": f"2 Monte Carlo steps of the 1024^2 lattice, one core (a single chain) ({wall:.1f} s)"}
    if workload == "fit":
        rate, units, wall = cpu_oracle_pool(_oracle_fit_chain, list(range(cores)), cores)
        return {"value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{cores} of the 128 chains of 256^2, 100 of the 2000 sweeps of a gradient step each, "
                          f"with per-sweep statistics ({wall:.1f} s wall)"}
    if workload == "triangular":
        import numpy as np
        per = 2
        rate, units, wall = cpu_oracle_pool(_oracle_tri, [(b * per, per) for b in range(cores)], cores)
        return {"value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{per * cores} of the 256 lattices, one sweep each ({wall:.1f} s wall)"}
    if workload == "nnn":
        per = max(1, 256 // cores)
        rate, units, wall = cpu_oracle_pool(_oracle_nnn, [(b * per, per) for b in range(cores)], cores)
        return {"value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{per * cores} of the 256 lattices, one sweep each ({wall:.1f} s wall)"}
    if workload == "few256":
        lats = few256()
        rate, units, wall = cpu_oracle_rate(lats, 40, min(cores, len(lats)))
        return {"value": rate, "unit": "site-updates/s", "cores": min(cores, len(lats)), "kind": "oracle",
                "sample": f"the 16 lattices x 40 sweeps ({wall:.1f} s wall)"}
    if workload == "ising_small":
        lats = wl.ising_small()
        rate, units, wall = cpu_oracle_rate(lats, 1000, min(cores, len(lats)))
        return {"value": rate, "unit": "site-updates/s", "cores": min(cores, len(lats)), "kind": "oracle",
                "sample": f"the whole job: 8 lattices x 1000 sweeps ({wall:.1f} s wall)"}
    if workload == "grad":
        from oracle import estimator
        rng = np.random.default_rng(0)
        st = np.stack([rng.integers(-65536, 65536, size=(128, 1000)),
                       rng.integers(0, 131072, size=(128, 1000))], axis=-1)
        t0 = time.perf_counter()
        for _ in range(3):
            for i in range(128):
                estimator.ising_grad(st[i:i + 1], 0.45, 1.0, 0.0, 65536)
        wall = (time.perf_counter() - t0) / 3
        return {"value": 128 * 1000 / wall, "unit": "samples/s", "cores": 1, "kind": "oracle",
                "sample": "estimator over 128 chains x 1000 recorded sweeps, per-chain gradients (numpy)"}
    if workload == "cpm_batch":
        per = 16
        rate, units, wall = cpu_oracle_pool(_oracle_cpm_batch, [(b * per, per) for b in range(cores)], cores)
        return {"value": rate, "unit": "copy-attempts/s", "cores": cores, "kind": "oracle",
                "sample": f"{per * cores} of the 4096 lattices, two Monte Carlo steps each ({wall:.1f} s wall)"}
    if workload == "spinglass":
        per = 32
        rate, units, wall = cpu_oracle_pool(_oracle_spinglass, [(b * per, per) for b in range(cores)], cores)
        return {"value": rate, "unit": "site-sweeps/s", "cores": cores, "kind": "oracle",
                "sample": f"{per * cores} of the 1024 lattices, one spin-value iteration each (relaxed sweep, "
                          f"energy, reverse pass, quantised step; float64) ({wall:.1f} s wall)"}
    if workload == "dmc":
        B, L, K = DMC_SHAPE
        per = 48
        rate, units, wall = cpu_oracle_pool(_oracle_dmc, [(b * per, per, L, K) for b in range(cores)], cores)
        return {"value": rate, "unit": "site-sweeps/s", "cores": cores, "kind": "oracle",
                "sample": f"{per * cores} of the {B} lattices, one iteration each (forward {K} sweep(s), loss, "
                          f"reverse pass; float64) ({wall:.1f} s wall)"}
    if workload == "mlp":
        from oracle import mlp as omlp
        rng = np.random.default_rng(0)
        P = {k: rng.normal(0, 0.3, size=sh) for k, sh in omlp.shapes().items()}
        X = rng.uniform(-1, 1, size=(10000, 3))
        T = rng.normal(size=(10000, 2))
        t0 = time.perf_counter()
        for _ in range(5):
            Y, c = omlp.forward(P, X, np.zeros(3), np.ones(3))
            omlp.backward(P, c, Y, T, np.ones(3))
        wall = (time.perf_counter() - t0) / 5
        return {"value": 10000 / wall, "unit": "samples/s", "cores": cores, "kind": "oracle",
                "sample": "forward + backward of 10^4 samples in float64 numpy (BLAS threads)"}
    return None


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, period_ms=100):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms", str(period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self):
        return time.perf_counter()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (t, l) in self.lines if t0 <= t <= t1] or [l for (_, l) in self.lines[-3:]]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            p = [x.strip() for x in r.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SECTIONS = {
    # kernel: (file, section start, section end, end of the part of internal.h it depends on)
    "ising_strip_kernel": ("sweep_ising.cu",
                           "// One 8-byte table entry at a shared-memory address.",   # + accept_site
                           "// Copy every lattice", "cudaError_t launch_ising_strip("),
    "dmc_step_kernel": ("dmc.cu", "// One whole optimisation iteration per lattice",
                        "// loss[lat] = sum (target - s)^2", "cudaError_t launch_dmc_step("),
    "potts_strip_kernel": ("sweep_potts.cu",
                           "// ------------------------------------------------------------ strip kernel",
                           "__global__ void __launch_bounds__(256) potts_plain_kernel(",
                           "cudaError_t launch_potts_strip("),
}

# the host code that cuts a kernel's launch into work items (its counters depend on it)
PLANNER_SECTIONS = {
    "ising_strip_kernel": ("// Ising strip items:", "// Work list of the batched launch"),
}


def kernel_source_hash(kernel="ising_strip_kernel"):
    """Hash of the source of one kernel's section of its .cu file, the strip
    helpers, the part of internal.h the kernel depends on (up to its launch
    declaration) and the host code that cuts its launch into items, so that
    counters taken on an unchanged kernel and work list stay valid while other
    code changes."""
    csrc = os.path.join(ROOT, "paper_2304_01772_gb300", "csrc")
    fname, a, b, hdr_end = KERNEL_SECTIONS.get(kernel, ("sweep_ising.cu", "", "", ""))
    text = open(os.path.join(csrc, fname)).read()
    if a and a in text and b in text:
        text = text[text.index(a):text.index(b)]
    hdr = open(os.path.join(csrc, "internal.h")).read()
    if hdr_end and hdr_end in hdr:
        hdr = hdr[:hdr.index(hdr_end)]
    h = hashlib.sha256(text.encode())
    h.update(hdr.encode())
    h.update(open(os.path.join(csrc, "strip.cuh"), "rb").read())
    if kernel in PLANNER_SECTIONS:   # how the launch's rows are cut into items
        pa, pb = PLANNER_SECTIONS[kernel]
        plan = open(os.path.join(csrc, "abi.cpp")).read()
        if pa in plan and pb in plan:
            h.update(plan[plan.index(pa):plan.index(pb)].encode())
    return h.hexdigest()[:16]


def ncu_value(kernel, workload, key):
    """A per-launch counter (`key`) of `kernel` from the committed ncu summary,
    or None if absent or taken on a different kernel source."""
    if not kernel:
        return None
    path = os.path.join(ROOT, "profiles", f"{kernel.replace('_kernel', '')}_{workload}.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash(kernel):
            return None
        return float(kv[key].split()[0])
    except (OSError, KeyError, ValueError):
        return None


def ncu_traffic(kernel, workload="uneven512"):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return ncu_value(kernel, workload, "dram_bytes_per_full_launch")


def issue_roofline(kernel, workload, launch_ms, sm_mhz):
    """The binding resource of the integer-bound sweep kernels: warp-instruction
    issue.  achieved = the launch's executed warp instructions (ncu
    smsp__inst_executed.sum of the same launch, current source) / its CUDA-event
    time; peak = SMs x 4 schedulers x one warp instruction per cycle x the SM
    clock sampled during the timed region."""
    import torch
    inst = ncu_value(kernel, workload, "warp_instructions_per_full_launch")
    if not inst or not launch_ms or not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 4 * sm_mhz * 1e6
    ach = inst / (launch_ms * 1e-3)
    return {"bound": "issue", "achieved": ach, "peak": peak, "unit": "warp-instructions/s", "frac": ach / peak,
            "instructions_per_launch": inst, "sm_mhz": sm_mhz,
            "peak_source": f"{sms} SMs x 4 schedulers x 1 warp instruction per cycle at the sampled clock"}


def rng_ceiling(draws_per_update, updates_per_s, peak_gbs, bytes_per_update=2.0):
    """The random-number ceiling of a sweep on this GPU: spin_philox_xor (the
    sweeps' own Philox4x32-10 code, reduced to a digest) over 2^28 blocks =
    2^30 draws, best of 5 launches by CUDA events.  An Ising update consumes
    one 32-bit draw, a Potts update two, so no sweep on this stream can update
    faster than draws/s / draws_per_update."""
    import torch
    import paper_2304_01772_gb300 as sm
    n = 1 << 28
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        sm.philox_xor(SEED, 0, 0, 0, 0, n, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(5):
        torch.cuda.synchronize()
        e0.record(stream)
        sm.philox_xor(SEED, 0, 0, 0, 0, n, out)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    draws = 4.0 * n / (best * 1e-3)
    ceil = draws / draws_per_update
    return {"draws_per_s": draws, "draws_per_update": draws_per_update, "ceiling_updates_per_s": ceil,
            "ceiling_frac_of_hbm": ceil * bytes_per_update / 1e9 / peak_gbs,
            "kernel_updates_per_s": updates_per_s,
            "kernel_frac_of_ceiling": (updates_per_s / ceil) if updates_per_s else None,
            "source": "spin_philox_xor over 2^28 Philox4x32-10 blocks, best of 5, CUDA events"}


def dist_setup(n):
    from paper_2304_01772_gb300.dist import rank_info
    if n <= 1 and "RANK" not in os.environ:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", rank=rank, world_size=world)
    return rank, world, dist


def max_over_ranks(x, dist):
    from paper_2304_01772_gb300.dist import max_over_ranks as _max
    return _max(x, dist, device="cuda")


def sum_over_ranks(xs, dist):
    """Element-wise sums of a list of integers over all ranks."""
    if dist is None:
        return [int(x) for x in xs]
    import torch
    t = torch.tensor([int(x) for x in xs], dtype=torch.int64, device="cuda")
    dist.all_reduce(t)
    return [int(v) for v in t.tolist()]


def barrier(dist):
    import torch
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()


# ----------------------------------------------------------------- arms
def run_reference(args):
    """The CPU oracle as it stands on the host cores, on the same metric: W
    warm-up and K timed steps, each step one sweep of a rotating window of the
    512 lattices from their random start, the window sized so that the whole
    run takes about SPINMC_REFERENCE_BUDGET_S seconds (default 150) and never
    more than one full sweep per step; the steps of each group run as one
    stream of tasks on all cores."""
    import multiprocessing as mp

    import oracle
    from paper_2304_01772_gb300 import workloads as wl
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return 0
    lats = wl.uneven512()
    total_sites = wl.site_count(lats)
    cores = os.cpu_count() or 1
    K, W = max(1, args.steps), max(0, args.warmup)
    budget = float(os.environ.get("SPINMC_REFERENCE_BUDGET_S", "150"))
    oracle.build()
    with mp.get_context("spawn").Pool(cores) as pool:
        # calibration: one sweep of the first lattices (about a tenth of the workload)
        calib, acc = [], 0
        for i, d in enumerate(lats):
            calib.append((i, d, SEED, 1))
            acc += d["L"] ** 2
            if acc >= total_sites // 10:
                break
        t0 = time.perf_counter()
        res = pool.map(_oracle_lattice, calib, chunksize=1)
        est_rate = sum(r[0] for r in res) / (time.perf_counter() - t0)
        target = min(total_sites, max(1, int(est_rate * budget / (K + W))))
        # the W warm-up and K timed steps are windows of the rotating order; each group
        # of steps is run as one stream of tasks (largest first, all cores busy: a step
        # is a unit of work, not a barrier), and the timed group gives time per step
        ptr = 0

        def windows(n):
            nonlocal ptr
            out = []
            for _ in range(n):
                acc = 0
                while acc < target:
                    i = ptr % len(lats)
                    out.append((i, lats[i], SEED, 1))
                    acc += lats[i]["L"] ** 2
                    ptr += 1
            return sorted(out, key=lambda a: -a[1]["L"])

        if W:
            pool.map(_oracle_lattice, windows(W), chunksize=1)
        tasks = windows(K)
        t0 = time.perf_counter()
        res = pool.map(_oracle_lattice, tasks, chunksize=1)
        timed_s = time.perf_counter() - t0
        timed_updates = sum(r[0] for r in res)
    rate = timed_updates / timed_s
    sample = (f"per step, one sweep of a rotating window of the 512 lattices from their random start, "
              f"about {target:.3g} of the {total_sites:.3g} sites; the {K} timed steps (after {W} warm-up) "
              f"run as one stream of tasks on all cores, {timed_s:.1f} s timed")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": timed_s * 1e3 / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    from paper_2304_01772_gb300 import workloads as wl

    lats_all = wl.uneven512()
    job_sites = wl.site_count(lats_all)     # sites of the whole job per sweep (strong scaling)
    lats = lats_all
    cpu = None
    rank0_single = args.gpus == 1 and int(os.environ.get("RANK", 0)) == 0
    if rank0_single and not args.no_cpu:
        # before the first GPU call: a process pool forked after it could hang
        cores = os.cpu_count() or 1
        rate, updates, wall = cpu_oracle_rate(lats_all, max(1, args.cpu_sweeps), cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"all 512 lattices, {max(1, args.cpu_sweeps)} sweep(s) each ({updates:.3e} updates, "
                         f"{wall:.1f} s wall)"}

    import torch
    import paper_2304_01772_gb300 as sm
    rank, world, dist = dist_setup(args.gpus)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream()
    from paper_2304_01772_gb300.dist import rank_lattices, rank_seed
    if args.scaling == "strong":
        # this rank's share; lattice_id = global index + 1 keeps every lattice's stream
        lats, _ = rank_lattices(lats_all, rank, world)
        seed = SEED
    else:
        seed = rank_seed(SEED, rank)
    sites = wl.site_count(lats)             # sites of this rank per sweep
    # units of the whole job per sweep: the batch (strong) or one batch per rank (weak)
    units = job_sites if args.scaling == "strong" else job_sites * world
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=seed, max_record=max(16, args.e2e_steps))
    launch = sim.get_launch() if args.no_tune else sim.autotune(sweeps_per_trial=4)
    sim.sweep(args.warmup)

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", 0)))
    time.sleep(0.3)
    # ---- timed region: batched, graph-replayed
    barrier(dist)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.perf_counter()
    e0.record(stream)
    sim.sweep(args.steps)
    e1.record(stream)
    barrier(dist)
    t_wall1 = time.perf_counter()
    launches = sim.gpu_launches
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    clk = clocks.summary(t_wall0, t_wall1)

    # ---- plain per-lattice launches on the same state, same results
    sim.set_launch(1, True, 0, 256)
    sim.sweep(2)
    barrier(dist)
    e0.record(stream)
    sim.sweep(args.plain_steps)
    e1.record(stream)
    barrier(dist)
    ms_plain = max_over_ranks(e0.elapsed_time(e1), dist)
    # ---- the batched form's own kernels, one launch per lattice (what batching the launches buys)
    sim.set_launch(3, True, launch["tile_rows"] or -1, max(256, launch["threads"]))
    sim.sweep(2)
    barrier(dist)
    e0.record(stream)
    sim.sweep(args.plain_steps)
    e1.record(stream)
    barrier(dist)
    ms_plain3 = max_over_ranks(e0.elapsed_time(e1), dist)
    sim.set_launch(launch["mode"], True, launch["tile_rows"] or -1, launch["threads"])

    # ---- kernel time of the batched sweep kernels (CUDA events in the library)
    nk = min(args.steps, 200)
    sim.profile(True, 2 * nk)
    sim.sweep(nk)
    prof = sim.profile_read()
    sim.profile(False)
    clocks.stop()

    # ---- end to end through the C ABI with host buffers.  Every step is a job:
    # upload the spins from pinned host memory, one sweep, read back the spins
    # and that sweep's statistics.  Three contexts on three streams, so the
    # upload of step k+1 overlaps the sweep and download of step k.
    import ctypes
    L = sm.lib()
    span = sim.spins.numel()
    host_in = torch.empty(span, dtype=torch.int8, pin_memory=True)
    host_in.copy_(sim.spins.cpu())
    NB = 3   # contexts in flight
    host_out = [torch.empty(span, dtype=torch.int8, pin_memory=True) for _ in range(NB)]
    sims = [sim] + [sm.Sim(sm.SPIN_ISING, lats, seed=seed + 7919 * b, max_record=4)
                    for b in range(1, NB)]
    for x in sims[1:]:
        x.set_launch(launch["mode"], True, launch["tile_rows"] or -1, launch["threads"])
    streams = [torch.cuda.Stream() for _ in range(NB)]
    d_stats = [torch.empty((1, len(lats), sim.width), dtype=torch.int64, device="cuda") for _ in range(NB)]
    h_stats = [torch.empty((1, len(lats), sim.width), dtype=torch.int64, pin_memory=True) for _ in range(NB)]

    # NB contexts round robin; copies in each direction run first in, first out across
    # the streams (an upload waits for the previous upload, a download for the previous
    # download), so step k's upload overlaps step k-1's download instead of sharing
    # bandwidth with another upload, and a stream's next upload does not wait for its
    # own download of NB steps ago
    ev_up = [torch.cuda.Event() for _ in range(NB)]
    ev_down = [torch.cuda.Event() for _ in range(NB)]

    # the same with one bit per spin on the host (spin_load_spins_packed /
    # spin_store_spins_packed: unpack and pack kernels around the sweep)
    nw = sim.packed_words
    pin_in = torch.empty(nw, dtype=torch.int32, pin_memory=True)
    pin_out = [torch.empty(nw, dtype=torch.int32, pin_memory=True) for _ in range(NB)]
    sim.store_spins_packed(pin_in)
    torch.cuda.synchronize()

    def e2e_step(k, packed):
        x, st = sims[k % NB], streams[k % NB]
        sp = ctypes.c_void_p(st.cuda_stream)
        if packed:
            # one call: upload the packed state, one sweep (recorded), download the packed state
            sm._check(L.spin_sweep_packed(x.ctx, pin_in.data_ptr(), pin_out[k % NB].data_ptr(), 1, 1, sp),
                      x.ctx, "sweep_packed")
            sm._check(L.spin_observables(x.ctx, ctypes.c_int64(x.n_records - 1), 1, d_stats[k % NB].data_ptr(),
                                         None, None, sp), x.ctx, "obs")
            with torch.cuda.stream(st):
                h_stats[k % NB].copy_(d_stats[k % NB], non_blocking=True)
            return
        if k > 0:
            st.wait_event(ev_up[(k - 1) % NB])
        if packed:
            sm._check(L.spin_load_spins_packed(x.ctx, pin_in.data_ptr(), sp), x.ctx, "load")
        else:
            sm._check(L.spin_load_spins(x.ctx, host_in.data_ptr(), sp), x.ctx, "load")
        ev_up[k % NB].record(st)
        sm._check(L.spin_sweep(x.ctx, 1, 1, sp), x.ctx, "sweep")
        if k > 0:
            st.wait_event(ev_down[(k - 1) % NB])
        if packed:
            sm._check(L.spin_store_spins_packed(x.ctx, pin_out[k % NB].data_ptr(), sp), x.ctx, "store")
        else:
            sm._check(L.spin_store_spins(x.ctx, host_out[k % NB].data_ptr(), sp), x.ctx, "store")
        ev_down[k % NB].record(st)
        sm._check(L.spin_observables(x.ctx, ctypes.c_int64(x.n_records - 1), 1, d_stats[k % NB].data_ptr(),
                                     None, None, sp), x.ctx, "obs")
        with torch.cuda.stream(st):
            h_stats[k % NB].copy_(d_stats[k % NB], non_blocking=True)

    def e2e_run(packed):
        for k in range(NB):
            e2e_step(k, packed)
        for st in streams:
            st.synchronize()
        barrier(dist)
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            e2e_step(k, packed)
        for st in streams:
            st.synchronize()
        barrier(dist)
        return max_over_ranks(time.perf_counter() - t0, dist)

    e2e_int8_s = e2e_run(False)
    e2e_s = e2e_run(True)
    st_host = h_stats[0]
    # host<->device bytes of one step of the whole job (every rank's copies)
    job_bytes = sum_over_ranks([4 * nw, 4 * nw + st_host.numel() * 8, span, span + st_host.numel() * 8], dist)

    if rank != 0:
        return 0
    value = units * args.steps / (ms * 1e-3)
    strip_ms = prof[1][0] / prof[1][1] if prof[1][1] else None
    rng = rng_ceiling(1, (sum(d["L"] ** 2 for d in lats if d["L"] in (512, 1024, 2048)) / (strip_ms * 1e-3))
                      if strip_ms else None, measured_peaks()[0])
    plain = units * args.plain_steps / (ms_plain * 1e-3)
    plain3 = units * args.plain_steps / (ms_plain3 * 1e-3)
    peak, peak_kind = measured_peaks()
    strip_sites = sum(d["L"] ** 2 for d in lats if d["L"] in (512, 1024, 2048))
    cls_sites = [sites - strip_sites, strip_sites]
    kernels = {}
    for cls, name in ((0, "ising_fused_kernel"), (1, "ising_strip_kernel")):
        kms, kn = prof[cls]
        if kn:
            b = 2.0 * cls_sites[cls]
            kernels[name] = {"launch_ms": kms / kn, "launches": kn, "algorithmic_bytes_per_launch": b,
                             "achieved_gbs": b / (kms / kn * 1e-3) / 1e9, "share_of_kernel_time": 0.0}
    overlapped = len(kernels) == 2   # the tile kernel runs on a side stream, concurrently with the strip kernel
    tot = sum(prof[c][0] for c in (0, 1)) or 1.0
    for cls, name in ((0, "ising_fused_kernel"), (1, "ising_strip_kernel")):
        if name in kernels:
            kernels[name]["share_of_kernel_time"] = prof[cls][0] / tot
    if overlapped:
        # its events then bracket co-running wall time, not its own cost; the ncu launch
        # list (serialised) gives its cost: about 0.023 ms per launch
        kernels["ising_fused_kernel"]["share_of_kernel_time"] = None
        kernels["ising_fused_kernel"]["stream"] = "side stream, overlaps ising_strip_kernel"
        kernels["ising_strip_kernel"]["share_of_kernel_time"] = None
    dom = ("ising_strip_kernel" if overlapped else
           (max(kernels, key=lambda k: kernels[k]["share_of_kernel_time"]) if kernels else None))
    achieved = kernels[dom]["achieved_gbs"] if dom else None
    alg_bytes = kernels[dom]["algorithmic_bytes_per_launch"] if dom else None
    kms_dom = kernels[dom]["launch_ms"] if dom else None
    kn = kernels[dom]["launches"] if dom else 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": args.scaling, "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattices": len(lats_all), "sites_per_sweep": job_sites,
                   "split": ("the batch split over the ranks by site count, lattice_id = global index + 1"
                             if args.scaling == "strong" else "every rank runs the whole batch, seed + rank"),
                   "rank0_lattices": len(lats), "rank0_sites_per_sweep": sites,
                   "launch": "batched work-list kernels, CUDA graph replay; autotuned form "
                             + json.dumps(launch),
                   "l2": "inputs larger than L2 (state 409 MB + ping-pong buffer), no flush",
                   "bit_exact": "spins identical to the CPU oracle and across launch forms (tests/)"},
        "plain": {"value": plain, "unit": UNIT, "steps": args.plain_steps,
                  "ms_per_step": ms_plain / args.plain_steps, "speedup_batched_vs_plain": value / plain,
                  "form": "two launches per lattice per sweep of the per-chunk plain kernel (launch mode 1)",
                  "same_kernels_per_lattice": {
                      "value": plain3, "unit": UNIT, "ms_per_step": ms_plain3 / args.plain_steps,
                      "speedup_batched_vs_this": value / plain3,
                      "form": "the batched form's kernels (row-strip for L >= 512, tile below) launched once "
                              "per lattice per sweep, each lattice cut into its own items (launch mode 3), "
                              "graph-replayed; identical spins (tests/test_gpu_parity.py)"}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": ncu_traffic(dom),
                     "kernel": dom, "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": kms_dom, "timed_launches": kn,
                     "peak_source": f"{peak_kind} hbm_gbs (copy)", "kernels": kernels,
                     "issue": issue_roofline(dom, "uneven512", kms_dom, clk.get("sm_mhz") if clk else None),
                     "rng": rng},
        "e2e": {"value": units * args.e2e_steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": job_bytes[0], "d2h_bytes_per_step": job_bytes[1],
                "transfer": "one bit per spin: spin_sweep_packed uploads the packed state from pinned host "
                            "memory, unpacks it into the ping-pong buffer, runs one recorded sweep into the "
                            "spin buffer, packs and downloads the new state; then that sweep's statistics",
                "pipeline": "three contexts on three streams, so one step's copies overlap another's sweep; "
                            "the int8 leg orders each direction's copies first in, first out",
                "int8_spins": {"value": units * args.e2e_steps / e2e_int8_s, "unit": UNIT,
                               "h2d_bytes_per_step": job_bytes[2], "d2h_bytes_per_step": job_bytes[3]}},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_secondary(args):
    """Other configurations, one JSON line each (not the headline metric):
    potts_q3 / potts_q8: 64 Potts lattices 1024^2 at beta_c(q) * [0.8, 1.2];
    cpm1024: cellular Potts 1024^2, 2000 cells (a step = one Monte Carlo step);
    ising_small: 8 Ising lattices 64^2, statistics recorded every sweep;
    few256: 16 Ising lattices 256^2, statistics recorded every sweep;
    grad: the fluctuation-estimator gradient over recorded statistics;
    mlp: one training step of the BF16 surrogate."""
    cpu = None if args.no_cpu else cpu_baseline_secondary(args.workload, os.cpu_count() or 1)
    import torch
    import paper_2304_01772_gb300 as sm
    from paper_2304_01772_gb300 import workloads as wl
    stream = torch.cuda.current_stream()
    if args.workload in ("grad", "mlp"):
        return run_grad_mlp(args, cpu)
    if args.workload == "dmc":
        return run_dmc(args, cpu)
    if args.workload == "fit":
        return run_fit(args, cpu)
    if args.workload == "spinglass":
        return run_spinglass(args, cpu)
    if args.workload == "cpm_batch":
        return run_cpm_batch(args, cpu)
    if args.workload == "rng":
        peak, kind = measured_peaks()
        r = rng_ceiling(1, None, peak)
        line = {"metric": "Philox4x32-10 draws/s (rng)", "value": r["draws_per_s"], "unit": "draws/s",
                "n_gpus": 1, "steps": 5, "warmup": 2, "higher_is_better": True, "dtype": "u32",
                "data": "synthetic", "config": {"workload": "rng: the sweeps' Philox4x32-10 stream alone, "
                                                            "2^28 blocks per launch reduced to an XOR digest"},
                "gpu_launches": 1, "rng": r}
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
        return 0
    record = False
    if args.workload.startswith("potts"):
        q = int(args.workload[-1])
        lats = wl.potts_batch(q)
        sim = sm.Sim(sm.SPIN_POTTS, lats, seed=SEED, max_record=16)
        units, unit = wl.site_count(lats), "site-updates/s"
        desc = f"64 q={q} Potts lattices 1024^2, beta = ln(1+sqrt(q)) * linspace(0.8, 1.2, 64), uint8"
    elif args.workload == "triangular":
        lats = [dict(L=192, beta=0.2 + 0.15 * k / 255, J=1.0, h=0.0, geometry=1) for k in range(256)]
        sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=16)
        units, unit = wl.site_count(lats), "site-updates/s"
        desc = ("256 triangular-lattice Ising lattices 192^2 (six neighbours, three colours), "
                "beta = linspace(0.2, 0.35, 256) across beta_c = ln(3)/4")
    elif args.workload == "nnn":
        lats = wl.nnn256()
        sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=16)
        units, unit = wl.site_count(lats), "site-updates/s"
        desc = ("256 Ising lattices 256^2 with first and second neighbours (four colours), J = 1, "
                "J2 ~ U(-0.5, 0.5), beta ~ U(0.2, 0.45), h ~ N(0, 0.05)")
    elif args.workload == "cpm1024":
        p = wl.cpm1024()
        sim = sm.Sim(sm.SPIN_CPM, [dict(L=p["L"])], seed=SEED, max_record=16,
                     cpm=dict(J=p["J"], **{"lambda": p["lam"]}, target=p["target"], n_cells=p["n_cells"],
                              T=p["T"], side=p["side"], cols=p["cols"]))
        units, unit = p["L"] ** 2, "copy-attempts/s"
        desc = "cellular Potts 1024^2, 2000 cells of 20x20, J=[[0,16,16],[16,2,11],[16,11,14]], A=400, lambda=1, T=10"
    elif args.workload == "few256":
        lats = few256()
        sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=args.steps)
        units, unit = wl.site_count(lats), "site-updates/s"
        record = True
        desc = "16 Ising lattices 256^2, beta = linspace(0.3, 0.55, 16), J = 1, h = 0, E and M recorded every sweep"
    else:
        lats = wl.ising_small()
        sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=args.steps)
        units, unit = wl.site_count(lats), "site-updates/s"
        record = True
        desc = "8 Ising lattices 64^2, beta = linspace(0.2, 0.6, 8), E and M recorded every sweep"
    launch = sim.get_launch() if (args.no_tune or args.workload == "cpm1024") else sim.autotune(4)
    sim.sweep(args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.sweep(args.steps, record=record)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    line = {"metric": f"{unit} ({args.workload})", "value": units * args.steps / (ms * 1e-3), "unit": unit,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "dtype": "uint8" if args.workload.startswith("potts") else
            ("int32" if args.workload == "cpm1024" else "int8"), "data": "synthetic",
            "config": {"workload": desc, "launch": launch}, "gpu_launches": sim.gpu_launches}
    if args.workload.startswith("potts"):
        nk = min(args.steps, 100)
        clocks = ClockSampler(0)
        time.sleep(0.3)
        tc0 = time.perf_counter()
        sim.profile(True, 2 * nk)
        sim.sweep(nk)
        prof = sim.profile_read()
        sim.profile(False)
        clk = clocks.summary(tc0, time.perf_counter())
        clocks.stop()
        cls = 1 if prof[1][1] else 0          # the strip kernel when the batch uses it
        kms, kn = prof[cls]
        kname = "potts_strip_kernel" if cls == 1 else "potts_fused_kernel"
        if kn:
            peak, kind = measured_peaks()
            ach = 2.0 * units / (kms / kn * 1e-3) / 1e9
            line["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                "traffic": ncu_traffic(kname, args.workload),
                                "kernel": kname, "launch_ms": kms / kn,
                                "note": "64 MiB state + partner ~ L2 size: largely L2-resident",
                                "peak_source": f"{kind} hbm_gbs",
                                "issue": issue_roofline(kname, args.workload, kms / kn,
                                                        clk["sm_mhz"] if clk else None),
                                "rng": rng_ceiling(2, units / (kms / kn * 1e-3), peak)}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def run_grad_mlp(args, cpu):
    """grad: the adjoint reduction (exact moments + FP64 covariance) over 128
    chains x 1000 recorded sweeps of 256^2 lattices (the fit's shape); mlp: one
    BF16 forward + backward of the surrogate on 10^4 samples."""
    import numpy as np
    import torch
    import paper_2304_01772_gb300 as sm
    from paper_2304_01772_gb300 import fit
    from paper_2304_01772_gb300 import workloads as wl
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    if args.workload == "grad":
        lats = wl.fit256()
        sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=1000)
        sim.sweep(1000, record=True)
        for _ in range(args.warmup):
            sim.grad(0, 1000)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            sim.grad(0, 1000, observable=0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        units, unit = 128 * 1000, "samples/s"
        desc = "fluctuation estimator d<E>/N / d(J, h) per chain: 128 chains of 256^2 x 1000 recorded sweeps"
    else:
        sur = fit.Surrogate(seed=3)
        X = torch.from_numpy(fit.sample_box(10000, seed=1)).cuda()
        T = torch.zeros((10000, 2), dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            sm.mlp_backward(sur.params, sur.mu, sur.inv_sigma, X, T)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            g, loss, _ = sm.mlp_backward(sur.params, sur.mu, sur.inv_sigma, X, T)
            sm.adam(sur.params, g, sur.m, sur.v, 1, 1e-3)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        units, unit = 10000, "samples/s"
        desc = "BF16 MLP 3-64-64-2: forward + backward + Adam on 10^4 samples (one training step)"
    line = {"metric": f"{unit} ({args.workload})", "value": units / (ms * 1e-3), "unit": unit, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "int64/fp64" if args.workload == "grad" else "bf16", "data": "synthetic",
            "config": {"workload": desc}}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def run_dmc(args, cpu):
    """Differentiable Monte Carlo pattern optimisation (Alg. 2): one step = one
    iteration of relaxed sweeps, pattern loss, reverse pass, Adam on the bond
    couplings and discretisation, for 1024 lattices of 64^2."""
    import torch
    from paper_2304_01772_gb300.dmc import PatternOptimizer
    B, L, K = DMC_SHAPE
    target = torch.from_numpy(dmc_targets(B, L)).cuda()
    opt = PatternOptimizer(target, beta=1 / 0.9, alpha=10.0, sweeps=K, seed=SEED, lr=5e-2)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        opt.step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        loss = opt.step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the fused kernel alone, and the same iteration as five separate launches
    def timed(fn, reps=20):
        fn()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps
    kernels = {}
    if opt.fused:
        kms = timed(opt.step)
        kernels["dmc_step_kernel"] = {"launch_ms": kms, "algorithmic_bytes_per_launch": 60 * B * L * L,
                                      "achieved_gbs": 60 * B * L * L / (kms * 1e-3) / 1e9,
                                      "bytes_per_site": "spins in + out, target, couplings and both Adam "
                                                        "moments in + out (2 bonds x 3 x 8 B)"}
    separate_ms = timed(opt.step_separate)
    top = max(kernels, key=lambda k: kernels[k]["launch_ms"])
    # the temperature study: coupling-gradient size of one iteration from the ordered start
    from paper_2304_01772_gb300.dmc import gradient_by_temperature
    temps = [0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0, 12.0, 20.0, 40.0]
    study = gradient_by_temperature(target, temps, alpha=10.0, sweeps=K, seed=SEED)
    peak, kind = measured_peaks()
    units = B * L * L * K
    separate = {"ms_per_step": separate_ms, "value": units / (separate_ms * 1e-3),
                "launches": "dmc_forward, dmc_loss, dmc_backward, adam, dmc_discretize (tape in HBM)"}
    line = {"metric": "site-sweeps/s (dmc)", "value": units / (ms * 1e-3), "unit": "site-sweeps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"differentiable Monte Carlo pattern optimisation: {B} Ising lattices of "
                                   f"{L}^2 with one coupling per bond, {K} relaxed sweep(s) per iteration, "
                                   "beta = 1/0.9, alpha = 10, h = 0, Adam lr 5e-2, striped/block targets; "
                                   "one step = forward + loss + reverse pass + Adam + discretisation",
                       "mean_loss_last_step": float(loss.mean()), "fused": opt.fused,
                       "separate_launches": separate,
                       "gradient_by_temperature": {
                           "T": temps, "mean_abs_dL_dJ": [g for _, g, _ in study],
                           "argmax_T": max(study, key=lambda r: r[1])[0],
                           "start": "couplings 1, spins all +1, one iteration per T"}},
            "roofline": {"bound": "hbm", "achieved": kernels[top]["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": kernels[top]["achieved_gbs"] / peak, "traffic": ncu_traffic(top, "dmc"), "kernel": top,
                         "peak_source": f"{kind} hbm_gbs", "kernels": kernels},
            "gpu_launches": (1 if opt.fused else 5) * args.steps}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def run_spinglass(args, cpu):
    """Energy minimisation over spin values on 1024 +-J spin glasses of 64^2:
    one step = one differentiable Monte Carlo iteration (relaxed sweep, energy
    and its gradient, reverse pass, quantised spin step, discretisation).  The
    final energies per spin of the three methods after equal iteration counts
    go in config."""
    import torch
    from paper_2304_01772_gb300.dmc import SpinOptimizer
    B, L = 1024, 64
    J = torch.from_numpy(spinglass_couplings(B, L)).cuda()
    g = torch.Generator().manual_seed(0)
    s0 = (torch.randint(0, 2, (B, L, L), generator=g).float() * 2 - 1).cuda()
    opt = SpinOptimizer(J, s0, seed=SEED)
    stream = torch.cuda.current_stream()
    opt.dmc(args.warmup, beta=2.0, alpha=10.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    trace = opt.dmc(args.steps, beta=2.0, alpha=10.0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    n_it = 60
    ann = SpinOptimizer(J, s0, seed=SEED).anneal([0.1 + 2.9 * k / (n_it - 1) for k in range(n_it)], 1)
    grd = SpinOptimizer(J, s0, seed=SEED).gradient(n_it)
    dmc = SpinOptimizer(J, s0, seed=SEED).dmc(n_it, beta=2.0, alpha=10.0)
    units = B * L * L
    line = {"metric": "site-sweeps/s (spinglass)", "value": units / (ms * 1e-3), "unit": "site-sweeps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"spin-value optimisation, {B} +-J spin glasses of {L}^2 (random bonds, "
                                   "random start); one step = one differentiable Monte Carlo iteration "
                                   "(relaxed sweep at beta 2, alpha 10, energy gradient, reverse pass, sign "
                                   "step eta 2, discretisation)",
                       "energy_per_spin_after_60_iterations": {
                           "annealed_metropolis_beta_0.1_to_3": float(ann[-1].mean()),
                           "gradient_only": float(grd[-1].mean()),
                           "dmc_best": float(dmc.min(axis=0).mean())},
                       "last_energy_per_spin": float(trace[-1].mean())},
            "gpu_launches": args.steps}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def run_cpm_batch(args, cpu):
    """The paper's cell-sorting setup (64^2, 36 cells + medium, T = 8, A = 25,
    lambda = 1) on 4096 lattices at once; one step = one Monte Carlo step of
    every lattice, all steps of the timed region in one launch."""
    import torch
    import paper_2304_01772_gb300 as sm
    from paper_2304_01772_gb300 import workloads as wl
    p = wl.cpm_paper()
    B = 4096
    batch = sm.CPMBatch(B, p["L"], dict(J=p["J"], **{"lambda": p["lam"]}, target=p["target"], n_cells=p["n_cells"],
                                        T=p["T"], side=p["side"], cols=p["cols"]), seed=SEED)
    stream = torch.cuda.current_stream()
    batch.run(args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # the same steps one launch each, with statistics recorded every step
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(20):
        batch.run(1, record=True)
    r1.record(stream)
    torch.cuda.synchronize()
    ms_rec = r0.elapsed_time(r1) / 20
    units = B * p["L"] ** 2
    line = {"metric": "copy-attempts/s (cpm_batch)", "value": units / (ms * 1e-3), "unit": "copy-attempts/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"batched cellular Potts, the paper's cell-sorting setup: {B} lattices of "
                                   "64^2, 36 cells of 5x5 + medium, J = [[0,16,16],[16,2,11],[16,11,14]], A = 25, "
                                   "lambda = 1, T = 8; all timed steps in one launch",
                       "one_launch_per_step_with_statistics_ms": ms_rec},
            "gpu_launches": 1}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def run_fit(args, cpu):
    """The differentiable fit at its stated size: 128 chains of 256^2 at beta =
    0.45, targets <E>/N = -1.2 and <M>/N = 0.5; a gradient step = 1000 burn-in
    + 1000 recorded sweeps, the fluctuation-estimator gradient and an Adam step.
    value = gradient steps per second; the BF16 surrogate (trained on 10^4
    chains of 64^2) and the steps to tolerance from the cold and the warm start
    go in config."""
    import torch
    from paper_2304_01772_gb300 import fit
    target, beta = (-1.2, 0.5), 0.45
    ens = fit.IsingEnsemble(128, 256, beta, seed=SEED, n_burn=1000, n_meas=1000)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fit.fit(ens, target, (1.0, 0.0), lr=1e-2, max_steps=args.warmup, tol=0.0)
    torch.cuda.synchronize()
    e0.record()
    fit.fit(ens, target, (1.0, 0.0), lr=1e-2, max_steps=args.steps, tol=0.0)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # per step: two sweep calls of 1000 sweeps (spin_gpu_launches counts the last call),
    # moments + pooling + expectations, two gradients (3 kernels each), one Adam step
    launches = args.steps * (2 * ens.sim.gpu_launches + 3 + 6 + 1)
    # surrogate warm start
    t0 = time.perf_counter()
    X = torch.from_numpy(fit.sample_box(10000, seed=1)).cuda()
    Y = fit.chain_targets(X, L=64, n_burn=300, n_meas=300)
    torch.cuda.synchronize()
    t_chains = time.perf_counter() - t0
    t0 = time.perf_counter()
    sur = fit.Surrogate(seed=3)
    n_tr = 9000                                   # the last 1000 chains are held out
    losses = sur.train(X[:n_tr].contiguous(), Y[:n_tr].contiguous(), epochs=1500, lr=3e-3)
    theta_w = [float(v) for v in sur.invert(target, beta).cpu()]
    t_train = time.perf_counter() - t0
    held = sur.predict(X[n_tr:].contiguous()) - Y[n_tr:]
    held_rmse = [float(v) for v in held.double().pow(2).mean(dim=0).sqrt().cpu()]
    runs = {}
    for name, th0 in (("cold", (1.0, 0.0)), ("warm", tuple(theta_w))):
        e = fit.IsingEnsemble(128, 256, beta, seed=SEED + 1, n_burn=1000, n_meas=1000)
        hist = []
        th, steps, loss = fit.fit(e, target, th0, lr=1e-2, max_steps=40, tol=2e-3, history=hist)
        runs[name] = {"steps": steps, "final_loss": loss, "theta": [float(v) for v in th.cpu()],
                      "mc_at_start": [hist[0][3], hist[0][4]]}
    xw = torch.tensor([[beta] + theta_w], dtype=torch.float32, device="cuda")
    warm_pred = [float(v) for v in sur.predict(xw)[0].cpu()]
    line = {"metric": "gradient steps/s (fit)", "value": 1e3 / ms, "unit": "gradient steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "dtype": "int8 spins, int64 moments, f64 covariance", "data": "synthetic",
            "config": {"workload": "differentiable fit: Ising 256^2, 128 chains, beta = 0.45, targets <E>/N = -1.2, "
                                   "<M>/N = 0.5; one step = 1000 burn-in + 1000 recorded sweeps, fluctuation "
                                   "gradient, Adam (lr 1e-2)",
                       "site_updates_per_step": 128 * 256 * 256 * 2000,
                       "launch": ens.sim.get_launch(),
                       "surrogate": {"chains": "10^4 (beta, J, h) from the box, 64^2, 300 + 300 sweeps; "
                                               "trained on 9000, the last 1000 held out",
                                     "chain_targets_s": t_chains, "train_1500_epochs_and_invert_s": t_train,
                                     "loss_first_last": [float(losses[0]), float(losses[-1])],
                                     "held_out_rmse_E_M": held_rmse,
                                     "warm_start_theta": theta_w,
                                     "warm_start_prediction_E_M": warm_pred,
                                     "warm_start_mc_E_M": runs["warm"]["mc_at_start"],
                                     "warm_start_error_vs_mc": [abs(a - b) for a, b in
                                                                zip(warm_pred, runs["warm"]["mc_at_start"])]},
                       "steps_to_loss_2e-3": runs},
            "gpu_launches": launches}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "uneven512":
        return run_secondary(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
