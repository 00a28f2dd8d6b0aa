#!/usr/bin/env python
"""Benchmark: grid points per second through descriptors -> LDOS -> integrals.

One step is one pass of the whole hot path over one snapshot: neighbour lists,
compute_ui, compute_zi/bi, the tcgen05 network, the DOS reduction, the FP64
Fermi-level bisection with the band energy, and the density pass (one
mala_predict call).  Default workload: Al fcc 4x4x4 (256 atoms, 16.2 A box) at
liquid-like disorder, 90^3 grid points, twojmax = 10 (91 descriptors), network
91 -> 400 -> 400 -> 250, 250 energies; synthetic inputs, random-init network.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload (the path needs
no exchange between replicas); rank 0 prints one JSON line with the
whole-job throughput (max time over ranks).  --impl reference times the FP64
CPU oracle on the host cores on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "grid points/s (descriptor+LDOS+density) & % roofline; p99 snapshot latency vs plain"
UNIT = "grid points/s"
WORKLOAD = ("Al fcc 4x4x4 (256 atoms, a=4.05 A, jitter N(0,0.3 A)), 90^3 = 729000 grid points, twojmax 10 "
            "(91 descriptors), rcut 4.676 A, MLP 91-400-400-250 LeakyReLU random-init, 250 energies at 0.1 eV, "
            "kT 0.0259 eV")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving trace (Poisson arrivals at 200/s; 0 skips the serving leg)")
    ap.add_argument("--serve-util-requests", type=int, default=300,
                    help="requests of the serving run at about 70%% utilisation")
    ap.add_argument("--serve-fp64-requests", type=int, default=24,
                    help="leading requests of the trace served by the plain FP64 path and, for the same "
                         "schedule, by the served mixed path")
    ap.add_argument("--workload-calls", type=int, default=2,
                    help="timed calls of the boron-cluster batch, Be slab and small FP64 legs (0 skips them)")
    ap.add_argument("--forces-calls", type=int, default=3,
                    help="timed calls of the band-energy forces leg (0 skips it)")
    ap.add_argument("--ace-calls", type=int, default=3, help="timed calls of the ACE descriptor leg (0 skips it)")
    ap.add_argument("--gauss-calls", type=int, default=3,
                    help="timed calls of the Gaussian descriptor leg (0 skips it)")
    ap.add_argument("--grid", type=int, default=0,
                    help="points per axis of the workload's grid (0: the workload's own 90; smaller grids are "
                         "for profiler captures, never for the bench line)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and self.uuid not in f[1]:
                continue
            rows.append(f)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower().startswith("active")})
        loaded = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload

def setup_workload(ctx, api, wl, torch, grid=0):
    snaps, bp, mlp, eg, _ = wl.config(2)
    snap = snaps[0]
    if grid:
        snap = wl.Snapshot(pos=snap.pos, species=snap.species, cell=snap.cell, grid=(grid, grid, grid),
                           periodic=snap.periodic)
    # input standardisation from the descriptors of this snapshot (model set-up)
    B = ctx.descriptors(snap, bp, api.MIXED).double()
    mlp = wl.with_input_scaling(mlp, B.mean(0).cpu().numpy(), 1.0 / (B.std(0).cpu().numpy() + 1e-12))
    del B
    model = api.Model(ctx, mlp)
    first = ctx.predict(snap, bp, model, eg, api.MIXED, n_electrons=0.0, raise_on_bracket=False)
    ne = ctx.electron_count(first["dos"], eg, 0.0)  # a reachable electron count: N(mu = 0)
    return snap, bp, mlp, model, eg, ne


def pct(v, q):
    v = sorted(v)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(np.ceil(q / 100.0 * len(v))) - 1))
    return v[k]


def _serve(ctx, api, trace, bp, model, eg, nes, time_scale=1.0):
    """Replay an arrival schedule through mala_submit/mala_poll (continuous batching over the
    serving slots): every request is submitted at its arrival time, completed tickets are read
    and released at once.  Latency = completion - arrival, queueing included."""
    lat, status, pending, i = [], [], {}, 0
    t0 = time.perf_counter()
    while i < len(trace) or pending:
        now = time.perf_counter() - t0
        while i < len(trace) and trace[i].arrival_s * time_scale <= now:
            tk = ctx.submit(trace[i].snapshot, bp, model, eg, api.MIXED, n_electrons=nes[i])
            pending[tk] = trace[i].arrival_s * time_scale
            i += 1
        for tk in list(pending):
            st = ctx.poll_status(tk)
            if st != 1:
                lat.append(time.perf_counter() - t0 - pending.pop(tk))
                status.append(st)
                ctx.release(tk)
        time.sleep(0.0002)
    return lat, status, time.perf_counter() - t0


def _plain_fp64(ctx, api, trace, bp, model, eg, nes):
    """The same schedule through the plain FP64 path, one snapshot at a time."""
    lat, status = [], []
    t0 = time.perf_counter()
    for i, rq in enumerate(trace):
        wait = rq.arrival_s - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        r = ctx.predict(rq.snapshot, bp, model, eg, api.FP64_PLAIN, n_electrons=nes[i], raise_on_bracket=False)
        status.append(r["status"])
        lat.append(time.perf_counter() - t0 - rq.arrival_s)
    return lat, status, time.perf_counter() - t0


def serving_leg(ctx, api, wl, mlp, bp, eg, n_req, n_util, n_fp64):
    """The serving trace (Poisson arrivals at 200/s; Al or Be bulk, 32..2048 atoms log-uniform,
    0.2 A spacing; network 91-400-400-250) served with mixed precision, at full size and at a
    rate giving about 70% utilisation, and its leading requests served by the plain FP64 path
    one snapshot at a time beside the served mixed path on the same schedule."""
    trace = wl.serving_trace(n_req, rate_per_s=200.0, seed=5)
    model = api.Model(ctx, mlp)
    # a reachable electron count per request: N(mu = 0) per unit volume of a calibration snapshot
    # of each material (untimed), times the request's volume
    per_vol = {}
    for mat in ("Al", "Be"):
        rq = next((r for r in trace if r.material == mat), None)
        if rq is None:
            continue
        r = ctx.predict(rq.snapshot, bp, model, eg, api.MIXED, n_electrons=0.0, raise_on_bracket=False)
        per_vol[mat] = ctx.electron_count(r["dos"], eg, 0.0) / rq.snapshot.volume
    nes = [per_vol[r.material] * r.snapshot.volume for r in trace]
    pts = [r.snapshot.n_points for r in trace]

    def summary(lat, status, span, n):
        ok = [l for l, st in zip(lat, status) if st in (0, -4)]
        return {"requests": n, "p50_ms": 1e3 * pct(lat, 50), "p99_ms": 1e3 * pct(lat, 99), "max_ms": 1e3 * max(lat),
                "points_per_s": sum(pts[:n]) / span, "wall_s": span,
                "unreachable_electron_count": int(sum(1 for st in status if st == -4)),
                "failed": int(sum(1 for st in status if st not in (0, -4))), "completed": len(ok)}

    out = {"trace": "Poisson arrivals at 200/s (seed 5), Al or Be (p = 1/2) at bulk density, N log-uniform in "
                    "[32, 2048] atoms, 0.2 A grid spacing; twojmax 10, network 91-400-400-250, 250 energies",
           "grid_points": int(sum(pts))}
    lat, st, span = _serve(ctx, api, trace, bp, model, eg, nes)
    out["served_mixed_200_per_s"] = summary(lat, st, span, len(trace))
    capacity = len(trace) / span  # requests/s the saturated run sustained
    rate = 0.7 * capacity
    if n_util > 0:
        sub = trace[:n_util]
        lat, st, span = _serve(ctx, api, sub, bp, model, eg, nes, time_scale=200.0 / rate)
        out["served_mixed_70pct_util"] = dict(summary(lat, st, span, len(sub)), rate_per_s=rate,
                                              note="arrival times of the trace scaled to 70% of the saturated "
                                                   "run's request throughput")
    if n_fp64 > 0:
        sub = trace[:n_fp64]
        ctx.predict(sub[0].snapshot, bp, model, eg, api.FP64_PLAIN, n_electrons=nes[0], raise_on_bracket=False)
        lat, st, span = _serve(ctx, api, sub, bp, model, eg, nes)
        out["subset_served_mixed"] = summary(lat, st, span, len(sub))
        lat, st, span = _plain_fp64(ctx, api, sub, bp, model, eg, nes)
        out["subset_plain_fp64_single"] = summary(lat, st, span, len(sub))
        out["subset"] = f"the first {len(sub)} requests of the trace, same arrival times, both arms"
    model.close()
    return out


def _kern(ctx, names):
    out = {}
    for k in names:
        t, n = ctx.profile_get(k)
        out[k] = {"ms": t, "launches": n}
    return out


def _leg_roofs(kern, roofline, P, pairs, twojmax, dims, n_e, fp32_peak, tensor_peak, hbm, fp64=False):
    """Rooflines of one call: algorithmic work of the call over the kernels' summed event time."""
    def ent(name, bound, work, peak, unit):
        t = kern[name]["ms"] / 1e3
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = work / t / scale if t > 0 else 0.0
        return {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak if peak else None,
                "work": work}
    r = {"k_zb": ent("k_zb", "alu", roofline.zb_flops_per_point(twojmax) * P, fp32_peak, "TFLOP/s"),
         "k_ui": ent("k_ui", "alu", roofline.ui_flops_per_point(twojmax, 1.0) * pairs, fp32_peak, "TFLOP/s"),
         "k_mlp": ent("k_mlp", "alu" if fp64 else "tensor", roofline.mlp_flops_per_point(dims) * P, tensor_peak,
                      "TFLOP/s"),
         "k_density": ent("k_density", "hbm", roofline.density_bytes(P, n_e, 8 if fp64 else 2, 8 if fp64 else 4), hbm,
                          "GB/s")}
    return r


def _timed_calls(torch, calls, fn):
    fn()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(calls):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / calls


def _reachable_ne(ctx, dos, eg):
    """N(mu = 0) of a DOS (the reading for random networks); if that count has no root on the
    bisection bracket (a random network's DOS can dip below zero), the midpoint of the counts
    at the bracket's ends, which always has one."""
    ne = ctx.electron_count(dos, eg, 0.0)
    lo = ctx.electron_count(dos, eg, eg.e0_eV - 20.0 * eg.kT_eV)
    hi = ctx.electron_count(dos, eg, eg.e0_eV + (eg.n_E - 1) * eg.de_eV + 20.0 * eg.kT_eV)
    if (lo - ne) * (hi - ne) < 0.0:
        return ne
    return 0.5 * (lo + hi)


def _pairs(ctx, snaps, rcut):
    return int(sum(int(ctx.neighbor_lists(s, rcut, cap=0)[0].sum().item()) for s in snaps))


KERNELS = ("k_neighbors", "k_ui", "k_zb", "k_mlp_in", "k_mlp", "k_dos_reduce", "k_sum_rows", "k_fermi", "k_density")


def workload_legs(ctx, api, wl, roofline, torch, calls, fp32_peak, fp64_peak, bf16_peak, hbm):
    """The paper-shaped workloads besides the default one, each through the public path:
    64 boron clusters in one mala_predict_batch, the Be slab with a stacking fault (streamed in
    chunks of tiles), and the small Al workload on the plain FP64 path."""
    out = {}
    # -- 64 boron clusters (8..96 atoms, 18 A box, 90^3 each), one batched call --
    try:
        snaps, bp, mlp, eg, _ = wl.config(3)
        B = ctx.descriptors_batch(snaps, bp, api.MIXED).double()
        mlp = wl.with_input_scaling(mlp, B.mean(0).cpu().numpy(), 1.0 / (B.std(0).cpu().numpy() + 1e-12))
        del B
        model = api.Model(ctx, mlp)
        first = ctx.predict_batch(snaps, bp, model, eg, api.MIXED, n_electrons=[0.0] * len(snaps),
                                  raise_on_bracket=False)
        nes = [_reachable_ne(ctx, r["dos"], eg) for r in first]
        P = sum(s.n_points for s in snaps)
        ms = _timed_calls(torch, calls, lambda: ctx.predict_batch(snaps, bp, model, eg, api.MIXED, n_electrons=nes,
                                                                  raise_on_bracket=False))
        ctx.profile(True)
        res = ctx.predict_batch(snaps, bp, model, eg, api.MIXED, n_electrons=nes, raise_on_bracket=False)
        kern = _kern(ctx, KERNELS)
        ctx.profile(False)
        pairs = _pairs(ctx, snaps, bp.rcut)
        out["boron_clusters"] = {
            "workload": "64 boron clusters, N ~ U{8..96} (seed 3), compact growth, 18 A periodic box, 90^3 each; "
                        "twojmax 10, network 91-400-400-11, 11 energies; one mala_predict_batch",
            "grid_points": P, "ms_per_call": ms, "grid_points_per_s": P / (ms / 1e3), "neighbour_pairs": pairs,
            "unreachable_electron_count": int(sum(1 for r in res if r["status"] == -4)), "kernels": kern,
            "rooflines": _leg_roofs(kern, roofline, P, pairs, bp.twojmax, mlp.dims, eg.n_E, fp32_peak, bf16_peak, hbm)}
        model.close()
    except Exception as e:  # reported, never costs the bench line
        out["boron_clusters"] = {"error": f"{type(e).__name__}: {e}"}
    # -- Be slab with a stacking fault: 16384 atoms, 183 x 317 x 336 grid --
    try:
        snaps, bp, mlp, eg, _ = wl.config(4)
        snap = snaps[0]
        B = ctx.descriptors(snap, bp, api.MIXED)
        mean = B.double().mean(0).cpu().numpy()
        std = B.double().std(0).cpu().numpy()
        del B
        mlp = wl.with_input_scaling(mlp, mean, 1.0 / (std + 1e-12))
        model = api.Model(ctx, mlp)
        r = ctx.predict(snap, bp, model, eg, api.MIXED, n_electrons=0.0, raise_on_bracket=False)
        ne = _reachable_ne(ctx, r["dos"], eg)
        P = snap.n_points
        ms = _timed_calls(torch, calls, lambda: ctx.predict(snap, bp, model, eg, api.MIXED, n_electrons=ne))
        ctx.profile(True)
        ctx.predict(snap, bp, model, eg, api.MIXED, n_electrons=ne)
        kern = _kern(ctx, KERNELS)
        ctx.profile(False)
        pairs = _pairs(ctx, [snap], bp.rcut)
        out["be_slab"] = {
            "workload": "hcp Be 16x16x16 orthohexagonal (16384 atoms) with one stacking fault, 10 A vacuum, "
                        f"grid {snap.grid[0]}x{snap.grid[1]}x{snap.grid[2]}; twojmax 10, rcut 4.5 A, "
                        "network 91-400-400-11, 11 energies; one mala_predict",
            "grid_points": P, "ms_per_call": ms, "grid_points_per_s": P / (ms / 1e3), "neighbour_pairs": pairs,
            "kernels": kern,
            "rooflines": _leg_roofs(kern, roofline, P, pairs, bp.twojmax, mlp.dims, eg.n_E, fp32_peak, bf16_peak, hbm)}
        model.close()
    except Exception as e:
        out["be_slab"] = {"error": f"{type(e).__name__}: {e}"}
    # -- small Al on the plain FP64 path --
    try:
        snaps, bp, mlp, eg, _ = wl.config(1)
        snap = snaps[0]
        B = ctx.descriptors(snap, bp, api.FP64_PLAIN)
        mlp = wl.with_input_scaling(mlp, B.mean(0).cpu().numpy(), 1.0 / (B.std(0).cpu().numpy() + 1e-12))
        model = api.Model(ctx, mlp)
        r = ctx.predict(snap, bp, model, eg, api.FP64_PLAIN, n_electrons=0.0, raise_on_bracket=False)
        ne = _reachable_ne(ctx, r["dos"], eg)
        P = snap.n_points
        ms = _timed_calls(torch, max(calls, 5), lambda: ctx.predict(snap, bp, model, eg, api.FP64_PLAIN,
                                                                    n_electrons=ne))
        ctx.profile(True)
        ctx.predict(snap, bp, model, eg, api.FP64_PLAIN, n_electrons=ne)
        kern = _kern(ctx, KERNELS)
        ctx.profile(False)
        pairs = _pairs(ctx, [snap], bp.rcut)
        out["al_small_fp64"] = {
            "workload": "Al fcc 2x2x2 (32 atoms, jitter N(0,0.1 A)), 18^3 grid, twojmax 6, network 30-100-100-11, "
                        "11 energies; plain FP64 path (mala_predict, MALA_FP64_PLAIN)",
            "grid_points": P, "ms_per_call": ms, "grid_points_per_s": P / (ms / 1e3), "neighbour_pairs": pairs,
            "kernels": kern,
            "rooflines": _leg_roofs(kern, roofline, P, pairs, bp.twojmax, mlp.dims, eg.n_E, fp64_peak, fp64_peak, hbm,
                                    fp64=True)}
        model.close()
    except Exception as e:
        out["al_small_fp64"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def forces_leg(ctx, api, roofline, model, snap, bp, eg, ne, calls, peak_tflops):
    """mala_band_forces (forward path + dE_b/dD + network backward + descriptor
    adjoint) on the bench workload: ms per call and the adjoint kernels' share."""
    import torch
    counts, _, _, _ = ctx.neighbor_lists(snap, bp.rcut, cap=0)
    pairs = int(counts.sum().item())
    P = int(np.prod(snap.grid))
    ctx.band_forces(snap, bp, model, eg, api.MIXED, n_electrons=ne)  # tables, workspaces
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(calls):
        out = ctx.band_forces(snap, bp, model, eg, api.MIXED, n_electrons=ne)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / calls
    ctx.profile(True)
    ctx.band_forces(snap, bp, model, eg, api.MIXED, n_electrons=ne)
    kern = {}
    for k in ("k_neighbors", "k_ui", "k_u_expand", "k_zb", "k_mlp_in", "k_mlp", "k_fermi", "k_egrad", "k_gemm_rows",
              "k_bwd_elementwise", "k_yi", "k_force"):
        t, n = ctx.profile_get(k)
        kern[k] = {"ms": t, "launches": n}
    ctx.profile(False)
    yi_f = roofline.yi_flops_per_point(bp.twojmax) * P
    fo_f = roofline.force_flops_per_pair(bp.twojmax) * pairs
    roof = {}
    for name, flops in (("k_yi", yi_f), ("k_force", fo_f)):
        t = kern[name]["ms"]  # one call's launches together do the call's work (k_yi: one launch per coupling group)
        ach = flops / (t / 1e3) / 1e12 if t > 0 else 0.0
        roof[name] = {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                      "frac": ach / peak_tflops, "flops": flops}
    F = out["forces"]
    return {"ms_per_call": ms, "grid_points_per_s": P / (ms / 1e3), "atoms": int(len(snap.pos)),
            "neighbour_pairs": pairs, "precision": "f32 descriptors/u/backward/adjoint, bf16 forward network, "
                                                   "f64 dE_b/dD, forces summed in 2^-40 fixed point",
            "max_abs_force_eV_per_A": float(np.max(np.abs(F))), "kernels": kern, "roofline": roof}


class AceSetting:
    """ACE descriptor set timed beside the bench workload: 401 columns (8 N = 1, 147 N = 2, 246 N = 3)."""
    rcut, n_species, nmax1, nmax2, lmax2, nmax3, lmax3 = 4.676, 1, 8, 6, 6, 3, 4


def ace_leg(ctx, api, roofline, snap, calls, peak_tflops):
    """mala_ace_descriptors on the bench snapshot: ms per call, points/s, k_ace's roofline."""
    import torch
    ap = AceSetting()
    counts, _, _, _ = ctx.neighbor_lists(snap, ap.rcut, cap=0)
    pairs = int(counts.sum().item())
    P = int(np.prod(snap.grid))
    out = ctx.ace_descriptors(snap, ap, api.MIXED)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(calls):
        ctx.ace_descriptors(snap, ap, api.MIXED, out=out)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / calls
    ctx.profile(True)
    ctx.ace_descriptors(snap, ap, api.MIXED, out=out)
    kern = {}
    for k in ("k_neighbors", "k_ace"):
        t, n = ctx.profile_get(k)
        kern[k] = {"ms": t, "launches": n}
    ctx.profile(False)
    flops = roofline.ace_flops(ap, pairs, P)
    # the kernel evaluates about half of the invariant terms (conjugate symmetry): the fraction
    # by the terms it executes is the one that measures the hardware
    fexe = roofline.ace_flops(ap, pairs, P, folded=True)
    t = kern["k_ace"]["ms"]
    ach = flops / (t / 1e3) / 1e12 if t > 0 else 0.0
    ach_exe = fexe / (t / 1e3) / 1e12 if t > 0 else 0.0
    return {"ms_per_call": ms, "grid_points_per_s": P / (ms / 1e3), "columns": int(out.shape[1]),
            "setting": {k: getattr(ap, k) for k in ("rcut", "n_species", "nmax1", "nmax2", "lmax2", "nmax3", "lmax3")},
            "neighbour_pairs": pairs, "kernels": kern,
            "roofline": {"k_ace": {"bound": "alu", "achieved": ach, "peak": peak_tflops, "unit": "TFLOP/s",
                                   "frac": ach / peak_tflops, "flops": flops,
                                   "flops_executed": fexe, "frac_executed": ach_exe / peak_tflops}}}


def gaussian_leg(ctx, api, snap, calls):
    """mala_gaussian_descriptors (rcut 4.676 A, sigma 0.5 A) on the bench snapshot: ms per call and
    grid points / neighbour pairs per second.  The work is the neighbour search itself (candidate
    tests per tile, FP64 only in the guard band), so no FLOP roofline is claimed.  A failure is
    reported under this key and never costs the bench line."""
    try:
        import torch
        rcut, sigma = 4.676, 0.5
        counts, _, _, _ = ctx.neighbor_lists(snap, rcut, cap=0)
        pairs = int(counts.sum().item())
        P = int(np.prod(snap.grid))
        out = ctx.gaussian_descriptors(snap, rcut, sigma, api.MIXED)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(calls):
            ctx.gaussian_descriptors(snap, rcut, sigma, api.MIXED, out=out)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / calls
        return {"ms_per_call": ms, "grid_points_per_s": P / (ms / 1e3), "neighbour_pairs": pairs,
                "pairs_per_s": pairs / (ms / 1e3), "rcut_A": rcut, "sigma_A": sigma}
    except Exception as e:  # reported, not raised
        return {"error": f"{type(e).__name__}: {e}"}


def kernel_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2411_19617_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# source files whose text decides each kernel's DRAM traffic (hashed against the ncu capture)
KERNEL_SOURCES = {
    "k_zb": ("snap_zb.cu", "snap_zb.cuh", "snap_pairs.cuh", "snap_common.cuh"),
    "k_ui": ("snap_ui.cu", "snap_common.cuh"),
    "k_mlp": ("mlp_tc.cu",),
    "k_density": ("integrate.cu",),
    "k_neighbors": ("snap_nbr.cu", "snap_common.cuh"),
}


def traffic_per_launch(kernel):
    """DRAM bytes (read + write) per launch of a kernel from the committed ncu
    summary profiles/traffic.json, if it was taken on the current kernel source;
    else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not t or t.get("kernel_hash") != kernel_hash(*KERNEL_SOURCES[kernel]):
        return None
    return t.get("dram_bytes_per_launch")


def rooflines(kernels, roofline, P, pairs, bp, dims, n_e, peaks, peak_src, fp32):
    """Roofline entry of every hot kernel: algorithmic work per launch (the
    definitions' counts, not the instruction stream) over the kernel's mean
    launch time from the library's CUDA events on the launching stream."""
    out = {}

    def entry(name, bound, work, peak, unit, source, **extra):
        t = kernels[name]["ms_per_launch"] / 1e3
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = work / t / scale if t > 0 else 0.0
        e = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak if peak else None,
             "traffic": traffic_per_launch(name), "work_per_launch": work, "peak_source": source}
        e.update(extra)
        out[name] = e

    fp32_peak, fp32_source = fp32
    zb_f = roofline.zb_flops_per_point(bp.twojmax)
    zb_full = roofline.zb_flops_per_point_full_count(bp.twojmax)
    entry("k_zb", "alu", zb_f * P, fp32_peak, "TFLOP/s", fp32_source,
          kernel="k_zb_units (compute_zi + compute_bi)", flop_per_point=zb_f,
          algorithmic_bytes=roofline.zb_bytes_per_point(bp.twojmax) * P,
          flop_per_point_full_count=zb_full,
          frac_full_count=(zb_full * P / (kernels["k_zb"]["ms_per_launch"] / 1e3) / 1e12) / fp32_peak,
          count_note=("flop_per_point: 10 per half-set coupling term with two nonzero Clebsch-Gordan factors, "
                      "j1 = j2 row pairs once, + 4 per half-set Z element; flop_per_point_full_count: every "
                      f"term of the full Z ({roofline.zi_terms_full(bp.twojmax)}) x 10 / 2 + 4 per full Z element"))
    entry("k_ui", "alu", roofline.ui_flops_per_point(bp.twojmax, 1.0) * pairs, fp32_peak, "TFLOP/s", fp32_source,
          kernel="k_ui (compute_ui, compensated sums)", flop_per_pair=roofline.ui_flops_per_point(bp.twojmax, 1.0),
          pairs=pairs)
    bf16 = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    entry("k_mlp", "tensor", roofline.mlp_flops_per_point(dims) * P, bf16, "TFLOP/s",
          f"{peak_src} bf16_tflops_sustained (cuBLAS bf16 GEMM, seconds-long loop)",
          kernel="k_mlp_tc (tcgen05 network + DOS partials)", flop_per_point=roofline.mlp_flops_per_point(dims))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    entry("k_density", "hbm", roofline.density_bytes(P, n_e), hbm, "GB/s", f"{peak_src} hbm_gbs (copy)",
          kernel="k_density (n(r), BF16 LDOS)", bytes_per_point=2 * n_e + 4)
    entry("k_neighbors", "hbm", roofline.neighbor_bytes(pairs, P), hbm, "GB/s", f"{peak_src} hbm_gbs (copy)",
          kernel="k_neighbors (neighbour records)", bytes_per_pair=20,
          note="bytes it must write (records and counts); the search itself is latency bound (FP64 tile set-up, "
               "candidate tests), so the fraction shows how far it is from the store stream")
    return out


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline / reference arm)

def oracle_sample(snap, bp, mlp_raw, eg, wl, n_points, nthreads, keep=None):
    """Time the oracle over n grid points of the workload: descriptors, network,
    DOS, Fermi level, band energy and density of the sample.  keep: a dict that
    receives the sample's points and oracle descriptors (after the clock stops)."""
    import oracle
    pts = wl.sample_points(snap.n_points, n_points, seed=1234)
    t0 = time.perf_counter()
    B = oracle.bispectrum_grid(snap, bp, points=pts, nthreads=nthreads)
    shift, scale = B.mean(axis=0), 1.0 / (B.std(axis=0) + 1e-12)
    L = oracle.mlp_forward(B, mlp_raw.W, mlp_raw.b, mlp_raw.leaky_slope, shift, scale)
    dV = snap.volume / snap.n_points
    D = oracle.dos(L, dV)
    ne = oracle.electron_count(D, 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    oracle.observables(L, dV, eg.e0_eV, eg.de_eV, eg.kT_eV, ne)
    t = time.perf_counter() - t0
    if keep is not None:
        keep["points"], keep["B"] = pts, B
    return t


def sample_size(snap, bp, mlp_raw, eg, wl, target_s, nthreads):
    """Points whose oracle run takes about target_s: fixed cost + per-point cost
    from two samples, the per-point cost never taken below half the larger
    sample's average (so timing noise cannot inflate the sample)."""
    n1, n2 = 256, 2048
    t1 = oracle_sample(snap, bp, mlp_raw, eg, wl, n1, nthreads)
    t2 = oracle_sample(snap, bp, mlp_raw, eg, wl, n2, nthreads)
    per_point = max((t2 - t1) / (n2 - n1), 0.5 * t2 / n2, 1e-9)
    fixed = max(t1 - n1 * per_point, 0.0)
    return int(min(snap.n_points, max(n1, (target_s - fixed) / per_point)))


def cpu_baseline(snap, bp, mlp_raw, eg, wl, target_s, keep=None):
    import oracle  # noqa: F401  (the CPU-baseline leg runs the oracle as it stands)
    nthreads = os.cpu_count() or 1
    n = sample_size(snap, bp, mlp_raw, eg, wl, target_s, nthreads)
    t = oracle_sample(snap, bp, mlp_raw, eg, wl, n, nthreads, keep=keep)
    return {"value": n / t, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{n} random grid points of the workload (descriptors, network, DOS, Fermi level, band energy, "
                      f"density of the sample), {t:.1f} s wall on {nthreads} threads"}


def descriptor_error(B_gpu, pts, B_ref):
    """FP32 descriptors against the FP64 oracle on the CPU-baseline sample:
    max |dB| / max(|B_ref|, floor) with the floor the component's RMS over the
    sample (the gated reading) and 1e-3 of it (reported, not gated)."""
    B = B_gpu[pts].double().cpu().numpy()
    rms = np.sqrt(np.mean(B_ref ** 2, axis=0))
    d = np.abs(B - B_ref)
    return {"points": int(len(pts)), "max_rel_rms_floor": float(np.max(d / np.maximum(np.abs(B_ref), rms))),
            "max_rel_1e-3_rms_floor": float(np.max(d / np.maximum(np.abs(B_ref), 1e-3 * rms))),
            "gate": "1e-5 at the RMS floor"}


# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle.build import build_oracle
    from paper_2411_19617_gb300 import workloads as wl
    build_oracle()
    snaps, bp, mlp, eg, _ = wl.config(2)
    snap = snaps[0]
    nthreads = os.cpu_count() or 1
    per_step_s = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    n = sample_size(snap, bp, mlp, eg, wl, per_step_s, nthreads)
    for _ in range(args.warmup):
        oracle_sample(snap, bp, mlp, eg, wl, n, nthreads)
    ts = [oracle_sample(snap, bp, mlp, eg, wl, n, nthreads) for _ in range(args.steps)]
    total = sum(ts)
    value = n * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_points_per_step": n, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"{n} random grid points of the workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2411_19617_gb300 import api, roofline, workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ctx = api.Context(local)
    snap, bp, mlp, model, eg, ne = setup_workload(ctx, api, wl, torch, args.grid)
    P = snap.n_points
    pairs = int(ctx.neighbor_lists(snap, bp.rcut, cap=0)[0].sum().item())  # (point, neighbour) pairs
    stream = torch.cuda.current_stream()

    def step(density_host=None, s=snap):
        return ctx.predict(s, bp, model, eg, api.MIXED, n_electrons=ne, density_host=density_host)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region (inputs resident; working set far above L2) ----
    props = torch.cuda.get_device_properties(local)
    uuid = str(getattr(props, "uuid", "") or "") or None
    clocks = ClockSampler(uuid)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    kernels = {}
    for k in ("k_neighbors", "k_ui", "k_zb", "k_mlp", "k_dos_reduce", "k_fermi", "k_density"):
        t, n = ctx.profile_get(k)
        kernels[k] = {"ms_per_launch": t / max(n, 1), "launches": n}
    _, launches = ctx.profile_get("all")
    ctx.profile(False)
    ms_max = ms
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    value = world * P * args.steps / (ms_max / 1e3)

    # ---- end to end through the public call with host buffers ----
    pos_pinned = torch.empty(snap.pos.shape, dtype=torch.float64, pin_memory=True).numpy()
    pos_pinned[:] = snap.pos
    sp_pinned = torch.empty(snap.species.shape, dtype=torch.int32, pin_memory=True).numpy()
    sp_pinned[:] = snap.species
    snap_h = wl.Snapshot(pos=pos_pinned, species=sp_pinned, cell=snap.cell, grid=snap.grid, periodic=snap.periodic)
    dens_pinned = torch.empty(P, dtype=torch.float32, pin_memory=True).numpy()
    step(dens_pinned, snap_h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    lat = []
    for _ in range(args.steps):
        a = time.perf_counter()
        r = step(dens_pinned, snap_h)
        lat.append(time.perf_counter() - a)
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * P * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(pos_pinned.nbytes + sp_pinned.nbytes),
           "d2h_bytes_per_step": int(dens_pinned.nbytes + 8 * eg.n_E + 8 * 9),
           "p50_latency_ms": 1e3 * statistics.median(lat), "max_latency_ms": 1e3 * max(lat)}

    # ---- rooflines of the hot kernels; the dominant one (compute_zi + compute_bi) heads the line ----
    peaks, peak_src = load_peaks()
    n_sms = int(props.multi_processor_count)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_scalar, fp32_packed, fp64_peak = ctx.measure_peaks()
    fp32_peak = max(fp32_scalar, fp32_packed)
    fp32 = (fp32_peak, f"measured FMA chains on every SM (scalar {fp32_scalar:.1f}, packed FP32x2 {fp32_packed:.1f} "
                       f"TFLOP/s; the larger); nominal {n_sms} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz = "
                       f"{roofline.fp32_peak_tflops(sm_max, n_sms):.1f}")
    roofs = rooflines(kernels, roofline, P, pairs, bp, mlp.dims, eg.n_E, peaks, peak_src, fp32)
    roof = dict(roofs["k_zb"])

    line = None
    if rank == 0:
        cpu = None
        derr = None
        if world == 1 and not args.no_cpu_baseline:
            keep = {}
            cpu = cpu_baseline(snap, bp, wl.config(2)[2], eg, wl, args.cpu_seconds, keep=keep)
            derr = descriptor_error(ctx.descriptors(snap, bp, api.MIXED), keep["points"], keep["B"])
        serving = None
        if world == 1 and args.serve_requests > 0:
            try:
                smlp = wl.config(5)[2]
                smlp = wl.MLP(dims=smlp.dims, W=smlp.W, b=smlp.b, leaky_slope=smlp.leaky_slope,
                              in_shift=mlp.in_shift, in_scale=mlp.in_scale)
                serving = serving_leg(ctx, api, wl, smlp, bp, eg, args.serve_requests, args.serve_util_requests,
                                      args.serve_fp64_requests)
            except Exception as e:  # reported, never costs the bench line
                serving = {"error": f"{type(e).__name__}: {e}"}
        workloads = None
        if world == 1 and args.workload_calls > 0:
            workloads = workload_legs(ctx, api, wl, roofline, torch, args.workload_calls, fp32_peak, fp64_peak,
                                      float(peaks.get("bf16_tflops_sustained", 1700.0)),
                                      float(peaks.get("hbm_gbs", 6800.0)))
        forces = None
        if world == 1 and args.forces_calls > 0:
            forces = forces_leg(ctx, api, roofline, model, snap, bp, eg, ne, args.forces_calls, fp32_peak)
        ace_res = None
        if world == 1 and args.ace_calls > 0:
            ace_res = ace_leg(ctx, api, roofline, snap, args.ace_calls, fp32_peak)
        gauss_res = None
        if world == 1 and args.gauss_calls > 0:
            gauss_res = gaussian_leg(ctx, api, snap, args.gauss_calls)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid_points": P, "precision":
                           "f32 descriptors (compensated neighbour sum), bf16 tcgen05 network with f32 accumulation, "
                           "f64 Fermi level and energy reductions",
                           "l2": "working set larger than L2 (u: 1.5 GB, neighbour records 0.9 GB, LDOS 0.36 GB)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": roof, "rooflines": roofs,
                "measured_peaks_tflops": {"fp32_scalar": fp32_scalar, "fp32_packed": fp32_packed, "fp64": fp64_peak,
                                          "sms": n_sms},
                "tuning": ctx.tuning_report().strip().splitlines(),
                "cpu_baseline": cpu, "descriptor_error": derr, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk, "kernels": kernels, "serving": serving, "workloads": workloads, "forces": forces,
                "ace": ace_res, "gaussian": gauss_res,
                "fermi_eV": r["fermi"], "band_energy_eV": r["band_energy"], "entropy_term_eV": r["entropy_term"]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
