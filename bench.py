"""Benchmark: PPN vs PN time steps on the twisting beam (20x20x80 vertices,
171,114 tets, E=1e6 Pa, nu=0.45, one end clamped, the other turned at 2 rad/s,
dt=1/30 s, tol 1e-4 relative gradient norm, FP32 bulk + FP64 reductions).

Prints ONE JSON line (rank 0).  A "step" is one backward-Euler time step: the
whole per-Newton-iteration pipeline (element evaluation, gradient, assembly,
PCG solves, PPN selection/projection/incremental update retries, line search,
update) until convergence.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (a deliberately slow program) on a
bounded sample of the same workload.  Multi-GPU runs are replicas (one scene
per rank, no exchange).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "twisting_beam_20x20x80", "n_verts": 32000, "n_tets": 171114, "E": 1e6,
            "nu": 0.45, "dt": 1.0 / 30.0, "omega_rad_s": 2.0, "tol": 1e-4, "tol_kind": "||g||2<=tol*||g0||2",
            "precision": "mixed: fp32 hessian/eigen/bsr/pcg, fp64 energy/gradient/norms/update"}


def build_spec():
    from ppn_inputs import twisting_beam_scene

    return twisting_beam_scene(20, 20, 80, h=0.01, E=1e6, nu=0.45, omega=2.0, dt=1.0 / 30.0, seed=0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    f, c = math.floor(k), math.ceil(k)
    return xs[f] if f == c else xs[f] + (xs[c] - xs[f]) * (k - f)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# Algorithmic bytes per unit of work (FP32 values, int32 indices), the scope table's
# per-unit figures:
#   K8 + K9, one CG iteration: per BSR block 36 B value + 4 B column; per row a 4 B
#            row pointer, 12 B of y, and ten 12-byte vector streams (x, r, z, p, q...)
#   K3, one assembly: per tet 16 blocks x 36 B of H^e read + 64 B of map; per BSR
#            block 36 B + 4 B written
#   K1, one element pass: per tet 16 B indices + 36 B D_m^-1 + 4 B volume read,
#            48 B g^e + 312 B packed H^e written; 24 B per vertex of unique
#            vertex data
def pcg_bytes_per_iter(info):
    return info["nnzb"] * 40 + info["n_verts"] * (16 + 10 * 12)


def assemble_bytes(info):
    return info["n_tets"] * (16 * 36 + 64) + info["nnzb"] * 40


def element_bytes(info):
    return info["n_tets"] * (16 + 36 + 4 + 48 + 312) + info["n_verts"] * 24


PCG_SOURCES = ("pcg_sr.cu", "pcg_common.cuh", "common.cuh", "kernels.h")
PCG_PROFILE = os.path.join(ROOT, "profiles", "k_pcg_sr_twisting_beam_20x20x80.json")


def pcg_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in PCG_SOURCES:
        with open(os.path.join(ROOT, "paper_2505_21013_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def pcg_profile_traffic():
    """DRAM bytes per launch of the resident PCG kernel from the ncu counters
    recorded beside its summary (profiles/*.json), or None when the kernel's
    sources changed since the capture."""
    try:
        kv = json.load(open(PCG_PROFILE))
        if kv.get("source_sha256_16") != pcg_source_hash():
            return None
        return {"bytes": float(kv["dram_bytes_per_launch"]), "cg_iters": int(kv["cg_iters_per_launch"])}
    except (OSError, ValueError, KeyError, TypeError):
        return None


def max_over_ranks(values, dist, device):
    """Element-wise max over ranks of this rank's timings (ms); identity at N=1."""
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def steps_per_s(world, steps, ms):
    """Whole-job throughput: every rank advances its own scene `steps` times
    (replicas, weak scaling) within the slowest rank's `ms`."""
    return world * steps / (ms / 1e3)


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    import paper_2505_21013_gb300 as P

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    spec = build_spec()
    total = args.warmup + args.steps
    # all steps' Dirichlet targets resident in HBM before the timed region
    tg = torch.tensor(np.stack([spec.targets_at(n) for n in range(total)]), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.Stream(device=dev)

    def run_mode(mode, profile):
        """W + K steps; per-step device time of the K timed steps.  With
        `profile`, per-kernel-family CUDA events are recorded too (an untimed
        run: the events add host work)."""
        sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
        sc.set_stream(stream.cuda_stream)
        info = sc.info()
        lat, stats, iters = [], [], []
        for n in range(total):
            timed = n >= args.warmup
            if timed and n == args.warmup:
                if dist:
                    dist.barrier()
                torch.cuda.synchronize()
                if profile:
                    sc.set_profiling(True)
            with torch.cuda.stream(stream):
                flush.zero_()
            sc.set_targets_device(tg[n].data_ptr())
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            rc, _, st = sc.step(mode, WORKLOAD["tol"], want_x=False)
            ev1.record(stream)
            if rc != 0:
                raise RuntimeError(f"step {n} returned status {rc}")
            if timed:
                ev1.synchronize()
                lat.append(ev0.elapsed_time(ev1))
                stats.append(st)
                iters.append(sc.iter_stats())
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        kt = sc.kernel_times() if profile else None
        cg = sum(it["cg_iters"] for its in iters for it in its)
        info = sc.info()  # with the layout of the last solve
        sc.close()
        return lat, stats, kt, info, cg

    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", 0)))
    sampler.start()
    lat_ppn, st_ppn, _, info, _ = run_mode(P.MODE_PPN, False)
    lat_pn, st_pn, _, _, _ = run_mode(P.MODE_PN, False) if not args.ppn_only else ([], [], None, None, 0)
    clocks = sampler.stop()
    # kernel breakdown: the same PPN steps again with per-family events
    _, _, kt, _, cg_total = run_mode(P.MODE_PPN, True)

    # end-to-end through the public API with host buffers: every step's targets
    # H2D from pinned host memory and its positions D2H into a pinned buffer, inside
    # the timed region
    sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
    tg_host = torch.from_numpy(np.stack([spec.targets_at(n) for n in range(total)])).pin_memory()
    out_host = torch.empty((spec.n_verts, 3), dtype=torch.float64).pin_memory()
    tg_np, out = tg_host.numpy(), out_host.numpy()
    e2e_ms = []
    for n in range(total):
        t0 = time.perf_counter()
        sc.set_targets(tg_np[n])
        rc, _, _ = sc.step(P.MODE_PPN, WORKLOAD["tol"], out=out)
        t1 = time.perf_counter()
        if rc != 0:
            raise RuntimeError(f"end-to-end step {n} returned status {rc}")
        if n >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    sc.close()

    ms_ppn, ms_pn, ms_e2e = max_over_ranks([sum(lat_ppn), sum(lat_pn), sum(e2e_ms)], dist, dev)
    K = args.steps
    value = steps_per_s(world, K, ms_ppn)

    # roofline of the dominant kernel family (by summed device time)
    peaks = measured_peaks()
    dom = max(kt.items(), key=lambda kv: kv[1]["total_ms"])
    name, rec = dom
    roof = None
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    if name == "pcg" and rec["launches"]:
        bpi = pcg_bytes_per_iter(info)
        iters_per_launch = cg_total / rec["launches"]
        alg_bytes = iters_per_launch * bpi
        avg_s = rec["total_ms"] / rec["launches"] / 1e3
        achieved = alg_bytes / avg_s / 1e9
        prof = pcg_profile_traffic()
        roof = {"bound": "hbm", "kernel": "k_pcg_sr (resident single-reduction block-Jacobi PCG)",
                "layout": P.PCG_LAYOUTS.get(info.get("pcg_layout", -1), "unknown"),
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": round(prof["bytes"]) if prof else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "bytes_per_cg_iter": bpi, "cg_iters_per_launch": iters_per_launch,
                "bytes_per_launch": alg_bytes, "avg_launch_ms": rec["total_ms"] / rec["launches"],
                "traffic_capture_cg_iters": prof["cg_iters"] if prof else None,
                "note": "achieved = algorithmic bytes (nnzb x 40 + n_verts x 136 per CG iteration) x CG iterations "
                        "per launch / average launch time; they are not DRAM bytes: the working set of one solve "
                        "stays L2-resident across iterations, so DRAM traffic is far below the algorithmic bytes "
                        "and the kernel is bound by grid-wide exchange latency"}
        # the other HBM-bound kernels of the step, on the same scope-table bytes
        kernels = {}
        for fam, fn, kname in (("assemble", assemble_bytes, "k_assemble"), ("element", element_bytes, "k_element")):
            k = kt.get(fam)
            if k and k["launches"]:
                ms = k["total_ms"] / k["launches"]
                gbs = fn(info) / (ms / 1e3) / 1e9
                kernels[kname] = {"bytes_per_launch": fn(info), "avg_launch_ms": round(ms, 5),
                                  "achieved": round(gbs, 1), "frac": round(gbs / peak, 4)}
        roof["kernels"] = kernels
    launches = int(sum(v["launches"] for v in kt.values()))
    r = {
        "value": value, "ms_per_step": ms_ppn / K,
        "p50_ms": percentile(lat_ppn, 0.5), "p99_ms": percentile(lat_ppn, 0.99),
        "ppn": {"newton_iters": sum(s["newton_iters"] for s in st_ppn),
                "projections": sum(s["total_projections"] for s in st_ppn),
                "cg_iters": sum(s["total_cg_iters"] for s in st_ppn),
                "attempts": sum(s["total_attempts"] for s in st_ppn)},
        "kernel_ms": {k: round(v["total_ms"], 3) for k, v in kt.items()},
        "roofline": roof, "clocks": clocks, "gpu_launches": launches,
        "e2e": {"value": steps_per_s(world, K, ms_e2e), "unit": "steps/s",
                "h2d_bytes_per_step": int(spec.fixed.size * 24), "d2h_bytes_per_step": int(spec.n_verts * 24)},
    }
    if lat_pn:
        r["pn"] = {"steps_per_s": steps_per_s(world, K, ms_pn), "ms_per_step": ms_pn / K,
                   "p50_ms": percentile(lat_pn, 0.5), "p99_ms": percentile(lat_pn, 0.99),
                   "newton_iters": sum(s["newton_iters"] for s in st_pn),
                   "projections": sum(s["total_projections"] for s in st_pn),
                   "cg_iters": sum(s["total_cg_iters"] for s in st_pn)}
        r["speedup_ppn_vs_pn"] = ms_pn / ms_ppn
    return r


VIOLENT = {"workload": "violent_twisting_beam_20x20x80", "E": 1e5, "nu": 0.45, "omega_rad_s": 20.0,
           "dt": 1.0 / 30.0, "tol": 1e-4}


def run_violent(steps=8, warmup=2):
    """The same 20x20x80 beam (171,114 tets), softer (E = 1e5) and turned at
    20 rad/s, so that the unprojected Hessian turns indefinite and PPN really
    selects, clamps and updates (Algorithm 1's inner loop).  PPN, PN and plain
    Newton from the same state: device time per step by CUDA events on the
    scene's stream (L2 flushed between steps), Newton iterations, projections,
    solves, selection ties, and per-kernel-family device time of the PPN steps
    (an untimed second pass with per-family events)."""
    import numpy as np
    import torch

    import paper_2505_21013_gb300 as P
    from ppn_inputs import twisting_beam_scene

    spec = twisting_beam_scene(20, 20, 80, h=0.01, E=VIOLENT["E"], nu=VIOLENT["nu"], omega=VIOLENT["omega_rad_s"],
                               dt=VIOLENT["dt"], seed=0)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tg = torch.tensor(np.stack([spec.targets_at(n) for n in range(warmup + steps)]), dtype=torch.float64,
                      device="cuda")

    def run(mode, profile=False):
        sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
        sc.set_stream(stream.cuda_stream)
        lat, agg = [], {"newton_iters": 0, "projections": 0, "attempts": 0, "cg_iters": 0, "ties": 0}
        for n in range(warmup + steps):
            if profile and n == warmup:
                torch.cuda.synchronize()
                sc.set_profiling(True)
            with torch.cuda.stream(stream):
                flush.zero_()
            sc.set_targets_device(tg[n].data_ptr())
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            rc, _, st = sc.step(mode, VIOLENT["tol"], want_x=False)
            ev1.record(stream)
            if rc != 0:
                raise RuntimeError(f"violent step {n} returned status {rc}")
            ev1.synchronize()
            if n >= warmup:
                lat.append(ev0.elapsed_time(ev1))
                agg["newton_iters"] += st["newton_iters"]
                agg["projections"] += st["total_projections"]
                agg["attempts"] += st["total_attempts"]
                agg["cg_iters"] += st["total_cg_iters"]
                agg["ties"] += st["n_ties"]
        kt = sc.kernel_times() if profile else None
        sc.close()
        r = {"steps_per_s": steps / (sum(lat) / 1e3), "ms_per_step": sum(lat) / steps,
             "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99), **agg,
             "projected_fraction": round(agg["projections"] / max(1, agg["newton_iters"] * spec.n_tets), 5)}
        return r, kt

    out = {"scene": VIOLENT["workload"], **{k: v for k, v in VIOLENT.items() if k != "workload"},
           "n_tets": spec.n_tets, "steps": steps, "warmup": warmup, "l2": "flushed between steps (256 MB write)"}
    out["ppn"], _ = run(P.MODE_PPN)
    out["pn"], _ = run(P.MODE_PN)
    out["newton"], _ = run(P.MODE_NEWTON)
    _, kt = run(P.MODE_PPN, profile=True)
    out["kernel_ms_ppn"] = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 3)} for k, v in kt.items()}
    out["speedup_ppn_vs_pn"] = out["ppn"]["steps_per_s"] / out["pn"]["steps_per_s"]
    out["speedup_ppn_vs_newton"] = out["ppn"]["steps_per_s"] / out["newton"]["steps_per_s"]
    return out


def profile_pcg(iters, repeats=4, workload="beam"):
    """Fixed-length PCG solves on the workload's assembled system (for ncu
    captures of the PCG kernel): one PPN step, then `repeats` solves of exactly
    `iters` CG iterations on the Hessian at that state.  workload "contact": the
    press scene (4 boxes of 40^3 vertices) at its initial pose, no step."""
    import numpy as np

    import paper_2505_21013_gb300 as P

    if workload == "contact":
        # the Hessian at the initial pose (K + M / dt^2; no PCG launch before the probes)
        from ppn_inputs import press_scene

        spec = press_scene(n=40, boxes=4, press_speed=0.05, dt=1.0 / 60.0, seed=0)
        sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
        sc.set_obstacles(spec.obstacles_at(-1))
        x = spec.rest
    else:
        spec = build_spec()
        sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
        sc.set_targets(spec.targets_at(0))
        rc, x, _ = sc.step(P.MODE_PPN, WORKLOAD["tol"], want_x=True)
        if rc != 0:
            raise RuntimeError(f"step returned status {rc}")
    nnzb = sc.info()["nnzb"]
    vals = sc.probe_assemble(x)
    b = np.random.default_rng(0).standard_normal((spec.n_verts, 3))
    b[spec.fixed] = 0
    out = []
    for _ in range(repeats):
        sc.set_profiling(True)  # resets the per-family CUDA-event times
        t0 = time.perf_counter()
        _, inf = sc.probe_pcg(vals, b, rel_tol=1e-30, max_iter=iters)
        dev = sc.kernel_times()["pcg"]["total_ms"]
        out.append({"iters": inf["iters"], "host_ms": (time.perf_counter() - t0) * 1e3, "device_ms": dev})
        sc.set_profiling(False)
    sc.close()
    print(json.dumps({"profile_pcg": out, "source_sha256_16": pcg_source_hash(), "nnzb": nnzb}))


def run_batched(n_scenes=64, steps=10, warmup=1, seed=0, tol=1e-4):
    """Batched workload: n independent cube/beam scenes (tet counts log-uniform in
    1k-50k, E log-uniform 1e4-1e7, nu in 0.3-0.48, dt in {1/30, 1/60, 1/120})
    advancing together, one launch per phase over all of them (ppn_step_batch).
    Returns scene-steps/s per mode, wall-clock around each batched step."""
    import paper_2505_21013_gb300 as P
    from ppn_inputs import random_batch_scenes

    specs = random_batch_scenes(n_scenes, seed=seed)
    out = {"n_scenes": n_scenes, "tets_total": int(sum(s.n_tets for s in specs)), "steps": steps}
    for name, mode in (("ppn", P.MODE_PPN), ("pn", P.MODE_PN)):
        scs = [P.Scene.from_spec(s, precision=P.PREC_MIXED) for s in specs]
        lat, newton, proj, capped = [], 0, 0, 0
        for n in range(warmup + steps):
            for sc, spec in zip(scs, specs):
                sc.set_targets(spec.targets_at(n))
            t0 = time.perf_counter()
            rc, st = P.ppn_step_batch(scs, [mode] * n_scenes, tol)
            dt = time.perf_counter() - t0
            if rc not in (0, P.ppn.PPN_ERR_NEWTON_MAXITER):
                raise RuntimeError(f"batched step {n} returned status {rc}")
            if n >= warmup:
                lat.append(dt * 1e3)
                newton += sum(x["newton_iters"] for x in st)
                proj += sum(x["total_projections"] for x in st)
                capped += sum(x["status"] == P.ppn.PPN_ERR_NEWTON_MAXITER for x in st)
        for sc in scs:
            sc.close()
        out[name] = {"scene_steps_per_s": n_scenes * steps / (sum(lat) / 1e3), "ms_per_batched_step": sum(lat) / steps,
                     "newton_iters": newton, "projections": proj, "steps_at_newton_cap": capped}
    out["speedup_ppn_vs_pn"] = out["ppn"]["scene_steps_per_s"] / out["pn"]["scene_steps_per_s"]
    # the linear solver's autotuner: per shape class the configuration it kept (layout x L2
    # priority of the streamed blocks, all bitwise-equal) and each one's time per CG iteration
    out["pcg_tuning"] = [{"tiles_per_cta": t["tiles_per_cta"], "blocks_per_row": t["blocks_per_row"],
                          "log2_matrix_mb": t["log2_matrix_mb"], "kept": t["kept"],
                          "us_per_iter": [round(x, 2) for x in t["us_per_iter"]]} for t in P.ppn.pcg_tuning()]
    return out


def run_serving(n_scenes=200, n_req=21000, warm=1000, rate_hz=500.0, seed=1, tol=1e-4, max_batch=64):
    """Request-stream workload: resident scenes of 2k-200k tets (log-uniform),
    admitted up to the server's HBM budget (80 % of the device), Poisson arrivals
    at rate_hz, each request one time step of a uniformly random scene, served
    with continuous batching (ppn_server_*).  A thread collects results in
    submission order while requests arrive.  Reports completed steps/s and
    p50/p99 latency (submit to result) over the requests after the first `warm`,
    per mode."""
    import queue
    import threading

    import numpy as np

    import paper_2505_21013_gb300 as P
    from ppn_inputs import poisson_arrivals, serving_scenes

    specs = serving_scenes(n_scenes, seed=seed)
    arrivals = poisson_arrivals(rate_hz, n_req, seed=seed)
    which = np.random.default_rng(seed).integers(0, n_scenes, size=n_req)
    out = {"n_scenes": n_scenes, "tets_total": int(sum(s.n_tets for s in specs)), "requests": n_req,
           "warmup_requests": warm, "rate_hz": rate_hz}
    for name, mode in (("ppn", P.MODE_PPN), ("pn", P.MODE_PN)):
        srv = P.Server(precision=P.PREC_MIXED, max_batch=max_batch)
        ids = [srv.add_scene(s) for s in specs]
        step_no = [0] * n_scenes
        pending = queue.Queue()
        results, errors = [], []

        def collect():
            while True:
                item = pending.get()
                if item is None:
                    return
                sid, t = item
                done, rc, _, stt, tm = srv.poll(t, sid)
                if rc not in (0, P.ppn.PPN_ERR_NEWTON_MAXITER):
                    errors.append(rc)
                results.append((sid, rc, stt, tm))

        th = threading.Thread(target=collect, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for a, k in zip(arrivals, which):
            now = time.perf_counter() - t0
            if a > now:
                time.sleep(a - now)
            k = int(k)
            pending.put((ids[k], srv.submit(ids[k], mode, tol, specs[k].targets_at(step_no[k]))))
            step_no[k] += 1
        pending.put(None)
        th.join()
        if errors:
            raise RuntimeError(f"serving requests failed with status {errors[:5]}")
        meas = results[warm:]
        lat = [tm["t_done_ms"] - tm["t_submit_ms"] for _, _, _, tm in meas]
        span = max(tm["t_done_ms"] for _, _, _, tm in meas) - min(tm["t_submit_ms"] for _, _, _, tm in meas)
        capped = {}
        for sid, rc, stt, _ in results:
            if rc:
                k = ids.index(sid)
                capped[specs[k].name] = {"tets": specs[k].n_tets, "E": specs[k].E, "nu": specs[k].nu,
                                         "dt": specs[k].dt, "grad_norm2": stt["final_grad_norm2"]}
        st = srv.stats()
        srv.close()
        out[name] = {"steps_per_s": 1e3 * len(meas) / span, "p50_ms": percentile(lat, 0.5),
                     "p99_ms": percentile(lat, 0.99), "mean_batch_max": float(np.mean([tm["batch_max"] for *_, tm in meas])),
                     "resident_scenes": st["resident_scenes"], "resident_gb": st["resident_bytes"] / 1e9,
                     "budget_gb": st["budget_bytes"] / 1e9, "requests_at_newton_cap": capped}
    out["speedup_ppn_vs_pn"] = out["ppn"]["steps_per_s"] / out["pn"]["steps_per_s"]
    return out


def run_ablation(steps=8, tol=1e-4):
    """Sensitivity of PPN to the tightening (alpha) and release (beta) rates of
    Sec. 4 on a violently twisted beam (10x10x40 vertices, E = 1e5, nu = 0.45,
    20 rad/s, dt = 1/30), where the unprojected Hessian turns indefinite: per
    (alpha, beta) the device time of `steps` time steps, Newton iterations,
    projected fraction and solves.  PN and plain Newton for reference."""
    import math

    import torch

    import paper_2505_21013_gb300 as P
    from ppn_inputs import twisting_beam_scene

    spec = twisting_beam_scene(10, 10, 40, h=0.02, E=1e5, nu=0.45, omega=20.0, dt=1.0 / 30.0, seed=0)

    def run(mode, alpha=0.5, beta=2.0):
        p = P.ppn_default_params()
        p.alpha, p.beta = alpha, beta
        sc = P.Scene.from_spec(spec, params=p, precision=P.PREC_MIXED)
        ms, newton, proj, att, cg, bad = 0.0, 0, 0, 0, 0, 0
        for n in range(steps):
            sc.set_targets(spec.targets_at(n))
            rc, _, st = sc.step(mode, tol, want_x=False)
            bad += rc != 0
            ms += st["device_ms"]
            newton += st["newton_iters"]
            proj += st["total_projections"]
            att += st["total_attempts"]
            cg += st["total_cg_iters"]
        sc.close()
        torch.cuda.synchronize()
        return {"alpha": alpha, "beta": beta, "ms": round(ms, 3), "newton_iters": newton,
                "projected_fraction": round(proj / max(1, newton * spec.n_tets), 5), "solves": att,
                "cg_iters": cg, "failed_steps": bad}

    grid = [run(P.MODE_PPN, a, b) for a in (0.01, 0.1, 0.25, 0.5, 0.75, 0.9)
            for b in (1.0, 2.0, 4.0, 16.0, math.inf)]
    best = min(grid, key=lambda r: r["ms"])
    default = next(r for r in grid if r["alpha"] == 0.5 and r["beta"] == 2.0)
    return {"scene": "twisting_beam_10x10x40_omega20", "n_tets": spec.n_tets, "steps": steps,
            "grid": grid, "pn": run(P.MODE_PN), "newton": run(P.MODE_NEWTON),
            "best": {"alpha": best["alpha"], "beta": best["beta"], "ms": best["ms"]},
            "default_over_best": round(default["ms"] / best["ms"], 3)}


def run_contact(steps=10, warmup=3, n=40, tol=1e-4):
    """Large contact-rich workload: 4 boxes of n^3 vertices side by side in a
    rigid analytic cylinder (radius 0.1 m) on the ground plane, under a press
    plane descending at 0.05 m/s, frictionless log-barrier contact (dhat = 1 mm),
    dt = 1/60, mixed precision.  Device time per step by CUDA events on the
    scene's stream (inputs resident; obstacle poses are a few hundred bytes
    per step), PPN and PN from the same initial state."""
    import torch

    import paper_2505_21013_gb300 as P
    from ppn_inputs import press_scene

    spec = press_scene(n=n, boxes=4, press_speed=0.05, dt=1.0 / 60.0, seed=0)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"scene": f"press_4x{n}^3", "n_verts": spec.n_verts, "n_tets": spec.n_tets, "steps": steps,
           "warmup": warmup, "dhat_m": 1e-3, "l2": "flushed between steps (256 MB write)"}

    def run(mode, profile=False):
        sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
        sc.set_stream(stream.cuda_stream)
        sc.set_obstacles(spec.obstacles_at(-1))
        lat, newton, proj, cg = [], 0, 0, 0
        for k in range(warmup + steps):
            if profile and k == warmup:
                torch.cuda.synchronize()
                sc.set_profiling(True)
            with torch.cuda.stream(stream):
                flush.zero_()
            sc.set_obstacles(spec.obstacles_at(k))
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            rc, x, st = sc.step(mode, tol, want_x=k == warmup + steps - 1)
            ev1.record(stream)
            if rc != 0:
                raise RuntimeError(f"contact step {k} returned status {rc}")
            ev1.synchronize()
            if k >= warmup:
                lat.append(ev0.elapsed_time(ev1))
                newton += st["newton_iters"]
                proj += st["total_projections"]
                cg += st["total_cg_iters"]
        info, kt = sc.info(), sc.kernel_times() if profile else None
        sc.close()
        r = {"steps_per_s": steps / (sum(lat) / 1e3), "ms_per_step": sum(lat) / steps,
             "p50_ms": percentile(lat, 0.5), "p99_ms": percentile(lat, 0.99), "newton_iters": newton,
             "projections": proj, "cg_iters": cg, "min_height_m": float(x[:, 1].min()),
             "top_m": float(x[:, 1].max()), "nnzb": info["nnzb"]}
        return r, info, kt

    out["ppn"], info, _ = run(P.MODE_PPN)
    out["pn"], _, _ = run(P.MODE_PN)
    # per-family device time of the same PPN steps (an untimed pass: the events add host work)
    prof, _, kt = run(P.MODE_PPN, profile=True)
    out["kernel_ms"] = {k: round(v["total_ms"], 3) for k, v in kt.items()}
    pcg = kt["pcg"]
    if prof["cg_iters"]:
        us = pcg["total_ms"] * 1e3 / prof["cg_iters"]
        peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
        gbs = pcg_bytes_per_iter(info) / (us * 1e-6) / 1e9
        out["pcg"] = {"launches": pcg["launches"], "cg_iters": prof["cg_iters"], "us_per_cg_iter": round(us, 2),
                      "algorithmic_gb_per_iter": round(pcg_bytes_per_iter(info) / 1e9, 4),
                      "achieved_gbs": round(gbs, 1), "hbm_frac_of_measured": round(gbs / peak, 4)}
    out["speedup_ppn_vs_pn"] = out["ppn"]["steps_per_s"] / out["pn"]["steps_per_s"]
    return out


def run_seeds(seeds=(0, 1, 2, 3, 4), steps=10, warmup=3, tol=1e-4):
    """The beam workload (20x20x80) for each jitter seed: PPN and PN device time of
    `steps` steps after `warmup`, per seed and summarised (the L2 is flushed
    between steps, as in the headline run)."""
    import torch

    import paper_2505_21013_gb300 as P
    from ppn_inputs import twisting_beam_scene

    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rows = []
    for seed in seeds:
        spec = twisting_beam_scene(20, 20, 80, h=0.01, E=1e6, nu=0.45, omega=2.0, dt=1.0 / 30.0, seed=seed)
        row = {"seed": seed}
        for name, mode in (("ppn", P.MODE_PPN), ("pn", P.MODE_PN)):
            sc = P.Scene.from_spec(spec, precision=P.PREC_MIXED)
            sc.set_stream(stream.cuda_stream)
            lat, newton, cg, proj = [], 0, 0, 0
            for n in range(warmup + steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                sc.set_targets(spec.targets_at(n))
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                rc, _, st = sc.step(mode, tol, want_x=False)
                ev1.record(stream)
                if rc != 0:
                    raise RuntimeError(f"seed {seed} step {n} returned status {rc}")
                ev1.synchronize()
                if n >= warmup:
                    lat.append(ev0.elapsed_time(ev1))
                    newton += st["newton_iters"]
                    cg += st["total_cg_iters"]
                    proj += st["total_projections"]
            sc.close()
            row[name] = {"steps_per_s": steps / (sum(lat) / 1e3), "p99_ms": percentile(lat, 0.99),
                         "newton_iters": newton, "cg_iters": cg, "projections": proj}
        row["speedup_ppn_vs_pn"] = row["ppn"]["steps_per_s"] / row["pn"]["steps_per_s"]
        rows.append(row)
    sp = [r["speedup_ppn_vs_pn"] for r in rows]
    v = [r["ppn"]["steps_per_s"] for r in rows]
    return {"workload": "twisting_beam_20x20x80 per seed", "steps": steps, "warmup": warmup, "seeds": rows,
            "ppn_steps_per_s": {"mean": statistics.mean(v), "min": min(v), "max": max(v)},
            "speedup_ppn_vs_pn": {"mean": statistics.mean(sp), "min": min(sp), "max": max(sp)}}


def host_cpu():
    """The host's logical CPU count and model name (for the oracle's timing)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        import platform

        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_sample(max_seconds=12.0, max_steps=3):
    """Time the FP64 oracle on the first PPN steps of the same beam (bounded), on all
    the host's cores (OpenMP over its independent element and SpMV-row loops) and on
    one core."""
    from oracle import oracle as O

    spec = build_spec()
    all_threads = max(1, os.cpu_count() or 1)

    def timed(threads):
        O.set_num_threads(threads)
        sc = O.Scene.from_spec(spec)
        t0 = time.perf_counter()
        n = 0
        while True:
            sc.set_targets(spec.targets_at(n))
            sc.step(O.PPN, WORKLOAD["tol"])
            n += 1
            if time.perf_counter() - t0 > max_seconds or n >= max_steps:
                break
        return n, time.perf_counter() - t0, O.num_threads()

    n_all, t_all, used = timed(all_threads)
    n_one, t_one, _ = timed(1)
    O.set_num_threads(all_threads)
    return {"value": n_all / t_all, "unit": "steps/s", "cores": used, "kind": "oracle",
            "sample": f"first {n_all} PPN time steps of the 20x20x80 twisting beam, FP64, {used} threads "
                      "(elements and SpMV rows in parallel)",
            "single_core": {"value": n_one / t_one, "unit": "steps/s", "cores": 1,
                            "sample": f"first {n_one} PPN time steps, one thread"}, **host_cpu()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ppn-only", action="store_true", help="skip the PN comparison run")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline beam only: skip the violent, batched, serving and contact sub-lines")
    ap.add_argument("--workload", default="beam",
                    choices=["beam", "batched", "serving", "ablation", "contact", "seeds", "violent"],
                    help="beam: the headline line; batched / serving: the multi-scene workloads; "
                         "ablation: the alpha/beta sweep; contact: boxes under a press in a cylinder; "
                         "seeds: the beam for jitter seeds 0-4")
    ap.add_argument("--profile-pcg", type=int, default=0, metavar="ITERS",
                    help="run fixed-length PCG solves for an ncu capture instead of the benchmark")
    args = ap.parse_args()
    if args.profile_pcg:
        profile_pcg(args.profile_pcg, workload=args.workload)
        return
    if args.workload != "beam" and args.impl == "ours":
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        if args.workload == "contact":
            r = run_contact(steps=args.steps, warmup=args.warmup)
        elif args.workload == "violent":
            r = run_violent(steps=args.steps, warmup=args.warmup)
        else:
            r = {"batched": run_batched, "serving": run_serving, "ablation": run_ablation,
                 "seeds": run_seeds, "violent": run_violent}[args.workload]()
        if int(os.environ.get("RANK", 0)) == 0:
            print(json.dumps({"workload": args.workload, **r}))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    base = {"metric": "time steps/s (PPN, twisting beam) with p50/p99 step latency, PPN vs PN at matched Newton tol",
            "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded Kuhn-grid beam; paper meshes unavailable)",
            "config": dict(WORKLOAD, l2="flushed between steps (256 MB write)",
                           parallelism="replicas" if args.gpus > 1 else "single")}

    if args.impl == "reference":
        if rank != 0:
            return
        per_step = []
        from oracle import oracle as O

        spec = build_spec()
        O.set_num_threads(max(1, os.cpu_count() or 1))
        sc = O.Scene.from_spec(spec)
        for n in range(args.warmup):
            pass  # the oracle has no warm-up effects; warm-up steps are not run to bound the time
        t_all = time.perf_counter()
        for n in range(args.steps):
            t0 = time.perf_counter()
            sc.set_targets(spec.targets_at(n))
            sc.step(O.PPN, WORKLOAD["tol"])
            per_step.append(time.perf_counter() - t0)
            if time.perf_counter() - t_all > 150:
                break
        k = len(per_step)
        v = k / sum(per_step)
        line = dict(base, impl="reference", value=v, ms_per_step=1e3 * sum(per_step) / k,
                    steps=k, p50_ms=1e3 * percentile(per_step, 0.5), p99_ms=1e3 * percentile(per_step, 0.99),
                    cpu_baseline={"value": v, "unit": "steps/s", "cores": O.num_threads(), "kind": "oracle",
                                  "sample": f"first {k} PPN steps of the beam (bounded to ~150 s), FP64, "
                                            f"{O.num_threads()} threads", **host_cpu()},
                    e2e={"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
        print(json.dumps(line))
        return

    dist = None
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
        dist = tdist
    r = run_ours(args, rank, world, dist)
    extras = {}
    if world == 1 and not args.no_extras:
        # the method's heuristic and the multi-scene and contact workloads on the same run,
        # each with its own device-timed figures (not the headline value)
        for key, fn in (("violent", lambda: run_violent(steps=8, warmup=2)),
                        ("batched", lambda: run_batched(n_scenes=64, steps=5, warmup=1)),
                        ("serving", lambda: run_serving(n_scenes=60, n_req=3000, warm=300, seed=1)),
                        ("contact", lambda: run_contact(steps=5, warmup=2))):
            t0 = time.perf_counter()
            extras[key] = fn()
            extras[key]["wall_s"] = round(time.perf_counter() - t0, 1)
    if rank == 0:
        line = dict(base, **r, **extras)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = oracle_sample()
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
