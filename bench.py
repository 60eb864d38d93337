#!/usr/bin/env python
"""Benchmark of the peridynamic stiffness product K u on one GB300.

Headline (one JSON line on stdout): K u throughput in GDOF/s on the 1024 x 1024
plate (delta = 3h, ~2.1M DOF per field), FP32, over a batch of independent
displacement fields (load cases) so that the inputs exceed L2 -- one step is one
batched K u launch through the C ABI.  Each rank of a multi-GPU launch works on
its own batch (weak scaling, no collective on the data path).

Also reported in the same line: the roofline of the dominant kernel, the SM
clocks seen during the timed region, an end-to-end figure with host buffers,
the FP32/FP64 x stencil/FFT x delta = 3h/6h variants, the static CG solve
(mixed precision vs FP64) to a relative residual of 1e-8, the paper's ADR
solver on the same plate and for the step counts of its 2D runs (also with the
surface correction), the 128^3 cube, the 2D crack loop and the notched 3D
block, and the CPU oracle timed on this host's cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--quick]
  python bench.py --case fft2d|stencil2d_f64|stencil3d|fft3d|crack|cg|adr|adr_mixed|sc|kw3d [--steps K] [--warmup W]
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "K·u GDOF/s (FP32, 1024x1024 plate, delta=3h)"
UNIT = "GDOF/s"
NSIDE, MH = 1024, 3
BATCH = 32          # 32 fields x 2 comps x 1M nodes x 4 B = 268 MB of inputs (> 129 MB L2)

# DRAM traffic of the dominant kernel per launch (ncu, dram__bytes_read.sum + dram__bytes_write.sum),
# recorded with the hash of the kernel sources it was taken on; reported only while they match.
TRAFFIC = {
    "kernel": "k_tbt2d_acc<3, 8> (64 x 64 tiles, difference form)",
    "sources": ["paper_2301_11828_gb300/csrc/pd_stencil2d_tma.cu", "paper_2301_11828_gb300/csrc/pd_tma2d.cuh",
                "paper_2301_11828_gb300/csrc/pd_stencil.cuh", "paper_2301_11828_gb300/csrc/pd_reduce.cuh"],
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch on 32 fields (the ncu capture
    # summarised under profiles/) divided by 32; valid while the sources hash to sha256
    "sha256": "3bcbc9f13d9aa152cd3985ed4356147885b2b0810ef576d0ed1416e2e62c2b34",
    "bytes_per_field": 15321312,
}


def _src_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, dev_uuid=None):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "50"]
        if dev_uuid:
            cmd.insert(1, f"--id={dev_uuid}")
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        time.sleep(0.12)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons, n = [], [], set(), 0
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            n += 1
            for name, val in zip(self.NAMES, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": n}


# --------------------------------------------------------------------------- helpers
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(value, dist, device):
    """Largest value over all ranks (the job's wall time is the slowest rank's); plain value at N=1."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _weak_value(dof_per_step, steps, world, elapsed_s):
    """Whole-job GDOF/s: every rank processes its own batch (weak scaling)."""
    return dof_per_step * steps * world / elapsed_s / 1e9


def _rank_seed(rank):
    """Each rank draws its own independent fields (load cases)."""
    return 2301_11828 + rank


def _time_fn(torch, fn, reps=20, warm=3):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps / 1e3   # seconds per call


def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _cpu_baseline(budget_s=10.0):
    """The oracle (FP64 direct bond sum, OpenMP) on one 1024^2 field, repeated for
    ~budget_s on all host cores, then timed once more on one core."""
    import numpy as np
    import oracle
    import synthetic as syn
    w = syn.large_plate(MH)
    al = oracle.alpha(2, w.E, w.delta)
    cores = oracle.threads()
    t0 = time.perf_counter()
    oracle.force(2, w.n, w.h, w.M, al, w.u)
    t1 = time.perf_counter() - t0
    reps = max(1, int(budget_s / max(t1, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.force(2, w.n, w.h, w.M, al, w.u)
    dt = (time.perf_counter() - t0) / reps
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.force(2, w.n, w.h, w.M, al, w.u)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    dof = 2 * w.N
    return {"value": dof / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} x K u on one 1024x1024 field (2.1M DOF), FP64 direct bond sum, "
                      f"{dt * 1e3:.1f} ms each on {cores} cores; once on 1 core: {dt1 * 1e3:.1f} ms",
            "one_core_value": dof / dt1 / 1e9, "cpu_model": _cpu_model()}


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import synthetic as syn
    w = syn.large_plate(MH)
    al = oracle.alpha(2, w.E, w.delta)
    for _ in range(args.warmup):
        oracle.force(2, w.n, w.h, w.M, al, w.u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.force(2, w.n, w.h, w.M, al, w.u)
    dt = time.perf_counter() - t0
    value = 2 * w.N * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "plate2d 1024x1024 delta=3h, K u, one field per step",
                                            "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": "one 1024x1024 field (2.1M DOF) per step, FP64 direct bond sum"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    import paper_2301_11828_gb300 as pd
    import synthetic as syn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pd.load_library()
    dev = torch.device("cuda", local)

    # ---- workload: B independent fields on the 1024^2 plate
    w = syn.large_plate(MH)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    B = args.batch
    base = torch.tensor(w.u, dtype=torch.float32, device=dev)
    U = torch.empty((B,) + base.shape, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(_rank_seed(rank))
    U.uniform_(-1.0, 1.0, generator=gen)
    U[0].copy_(base)
    OUT = torch.empty_like(U)
    flags = pd.PD_F32 | pd.PD_METHOD_STENCIL
    lib = pd.load_library()
    stream = torch.cuda.current_stream()
    sptr = pd._stream(stream)
    hdl = g.handle

    def step():
        rc = lib.pd_matvec_batch(hdl, B, pd._dptr(U), pd._dptr(OUT), flags, sptr)
        if rc:
            raise pd.PDError(rc, pd.pd_last_error())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    time.sleep(0.15)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_s, t_e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_s.record()
    for k in range(args.steps):
        evs[k][0].record()
        step()
        evs[k][1].record()
    t_e.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed = t_s.elapsed_time(t_e) / 1e3
    elapsed = _max_over_ranks(elapsed, dist, dev)
    if dist:
        dist.barrier()
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    dof_step = B * 2 * w.N
    value = _weak_value(dof_step, args.steps, ws, elapsed)

    # ---- roofline of the dominant kernel (the stencil launch is the whole step)
    peak, peak_kind = _peaks()
    alg_bytes = B * w.N * 2 * 2 * 4          # read u, write K u, FP32, 2 components
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    traffic = None
    if TRAFFIC["sha256"] and TRAFFIC["sha256"] == _src_hash(TRAFFIC["sources"]) and TRAFFIC["bytes_per_field"]:
        traffic = TRAFFIC["bytes_per_field"] * B
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": TRAFFIC["kernel"], "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes}

    # ---- end to end through the C ABI with pinned host buffers: pd_matvec_batch_host uploads,
    # multiplies and downloads chunks of the batch on three streams (copies overlapped)
    Uh = U.cpu().pin_memory()
    OUTh = torch.empty_like(Uh).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    uh_ptr, oh_ptr = pd._hptr(Uh), pd._hptr(OUTh)

    def e2e_step():
        rc = lib.pd_matvec_batch_host(hdl, B, uh_ptr, oh_ptr, flags, sptr)
        if rc:
            raise pd.PDError(rc, pd.pd_last_error())

    e2e_s = _time_fn(torch, e2e_step, reps=e2e_steps, warm=2)
    e2e = {"value": dof_step / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": Uh.numel() * 4,
           "d2h_bytes_per_step": OUTh.numel() * 4}
    del Uh, OUTh

    parity = None
    if rank == 0 and not args.no_parity:
        parity = _headline_parity(torch, pd, w, g, U, OUT, B)

    extras = {}
    if rank == 0 and not args.quick:
        extras = _extras(torch, pd, syn, dev)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = _cpu_baseline(args.cpu_budget)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"plate2d {NSIDE}x{NSIDE} delta=3h, K u on a batch of {B} fields "
                                       f"(load cases), one batched launch per step",
                           "global_batch": B * ws, "dof_per_field": 2 * w.N, "method": "stencil",
                           "l2": f"no flush: inputs {B * 2 * w.N * 4 / 1e6:.0f} MB > 129 MB L2",
                           "parallelism": f"replicas x{ws} (independent batches)"},
                "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": args.steps,
                "cpu_baseline": cpu, "parity_vs_oracle": parity}
        line.update(extras)
        print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _smooth_fields(n):
    """Smooth displacement fields (one to one-and-a-half waves across the plate),
    without and with a large constant part."""
    import numpy as np
    x = (np.arange(n[0]) + 0.5) / n[0]
    y = (np.arange(n[1]) + 0.5) / n[1]
    a = np.sin(2 * np.pi * x)[None, :] * np.cos(np.pi * y)[:, None]
    b = np.cos(3 * np.pi * x)[None, :] * np.sin(2 * np.pi * y)[:, None]
    return [np.stack([a, b]), np.stack([1.0 + 0.3 * a, 0.7 + 0.2 * b])]


def _rel(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _headline_parity(torch, pd, w, g, U, OUT, B):
    """Error of the timed product against the FP64 oracle (CPU, after the timed
    region): three of the timed fields as the last step left them, and the same
    launch on smooth fields with and without a constant part."""
    import oracle
    al = oracle.alpha(2, 1.0, w.delta)
    torch.cuda.synchronize()
    errs = {}
    for b in (0, B // 2, B - 1):
        ref = oracle.stiffness(2, w.n, w.h, w.M, al, U[b].double().cpu().numpy())
        errs[b] = _rel(OUT[b].double().cpu().numpy(), ref)
    sm = torch.tensor(_smooth_fields(w.n), dtype=torch.float32, device=U.device)
    out = torch.empty_like(sm)
    pd.pd_matvec_batch(g.handle, 2, sm, out, pd.PD_F32 | pd.PD_METHOD_STENCIL)
    torch.cuda.synchronize()
    serr = [_rel(out[i].double().cpu().numpy(),
                 oracle.stiffness(2, w.n, w.h, w.M, al, sm[i].double().cpu().numpy())) for i in range(2)]
    return {"timed_fields_rel_l2": {str(k): v for k, v in errs.items()}, "max_rel_l2": max(errs.values()),
            "smooth_fields_rel_l2": serr, "tolerance": 2e-5}


def _true_residual(oracle, dim, w, x, b, cons, al):
    """||P (b - K x)|| / ||P b|| with the oracle's FP64 operator (P K P)."""
    import numpy as np
    P = 1 - cons if cons is not None else 1.0
    r = b * P - oracle.stiffness(dim, w.n, w.h, w.M, al, x, cons=cons)
    return float(np.linalg.norm(r) / np.linalg.norm(b * P))


def _cufft_comparison(torch, pd, syn, dev, oracle):
    """cuFFT (torch.fft) with a whole-grid circulant embedding -- the comparison
    baseline for the FFT route (Algorithm 3 / 4) -- beside the library's own FFT
    tiles and stencils, on the 1024^2 plate (delta = 3h, 6h) and the 128^3 cube."""
    from paper_2301_11828_gb300.compare_cufft import CufftProduct
    res = {}
    for M in (3, 6):
        w = syn.large_plate(M)
        g = pd.Grid(2, w.n, w.h, w.M)
        al = oracle.alpha(2, 1.0, w.delta)
        for dt, name, B in ((torch.float32, "f32", 8), (torch.float64, "f64", 4)):
            U = torch.rand((B, 2, NSIDE, NSIDE), dtype=dt, device=dev) * 2 - 1
            cp = CufftProduct(g, dt)
            t = _time_fn(torch, lambda: cp(U), reps=5)
            out = cp(U)
            torch.cuda.synchronize()
            ref = oracle.stiffness(2, w.n, w.h, w.M, al, U[0].double().cpu().numpy())
            res[f"plate1024_M{M}_{name}"] = {"gdofs": round(B * 2 * w.N / t / 1e9, 2), "L": list(cp.L),
                                             "rel_l2_vs_oracle": _rel(out[0].double().cpu().numpy(), ref)}
            del U, out, cp
        g.close()
    w = syn.cube(128, 3)
    g = pd.Grid(3, w.n, w.h, w.M)
    U = torch.tensor(w.u, dtype=torch.float32, device=dev)[None]
    cp = CufftProduct(g, torch.float32)
    t = _time_fn(torch, lambda: cp(U), reps=5)
    out = cp(U)
    torch.cuda.synchronize()
    ref = oracle.stiffness(3, w.n, w.h, w.M, oracle.alpha(3, 1.0, w.delta), U[0].double().cpu().numpy())
    res["cube128_M3_f32"] = {"gdofs": round(3 * w.N / t / 1e9, 2), "L": list(cp.L),
                             "rel_l2_vs_oracle": _rel(out[0].double().cpu().numpy(), ref)}
    del U, out, cp
    g.close()
    return res


def _crack512(torch, pd, syn, dev, oracle, nsteps=2000):
    """The 2D pre-cracked plate of Sec. 5.2 at its stated size: 512^2, delta = 3h,
    s0 = 1e-3, rho = 1, lognormal modulus, centre pre-notch, tensile edge
    velocity; Algorithm 2 for 2000 steps at dt = 0.8 x the stable step of the
    actual field (pd_stable_dt); then the gradient of L = 1/2 |u_final|^2 with
    respect to the modulus field by the checkpointed adjoint of the same 2000
    steps.  Timed after warm-up runs; the first 100 steps are checked against
    the oracle's Verlet loop from the same state."""
    import numpy as np
    from paper_2301_11828_gb300.autograd import verlet_run
    w = syn.crack_plate(512, 3)
    lay = w.extra["vel_layers"]
    cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
    cons[1] = lay != 0
    vp = np.zeros((2,) + lay.shape)
    vp[1] = lay * w.extra["v0"]
    E_np = w.extra["E_field"]
    Et = torch.tensor(E_np, device=dev)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=cons, E_field=Et, s0=w.s0)
    notch = g.break_segment(w.extra["notch"], w.extra["notch_den"])
    mask0 = g.bond_mask().clone()
    dt = 0.8 * g.stable_dt()
    vpt = torch.tensor(vp, device=dev)
    v_init = np.where(cons != 0, vp, w.extra["v_ramp"])   # the ramp inside, the layers' velocity on them
    v0t = torch.tensor(v_init, device=dev)
    res = {"steps": nsteps, "dt": dt, "stable_dt": dt / 0.8, "E_max": float(E_np.max()), "notch_bonds": notch,
           "initial_velocity": "uniform stretch rate (v0 (2y/L - 1)), edge layers at +-v0"}
    # warm-up on the same grid (workspaces, the adjoint's segment buffers), then the bond state reset
    u = torch.zeros((2,) + lay.shape, dtype=torch.float64, device=dev)
    v = v0t.clone()
    g.step(u, v, None, nsteps=5, dt=dt, v_prescribed=vpt)
    E = Et.clone().requires_grad_(True)
    uN = verlet_run(g, E, torch.zeros_like(u), v0t.clone(), 50, dt, v_prescribed=vpt, checkpoint_every=45)
    (0.5 * (uN * uN).sum()).backward()
    g.set_bond_mask(mask0)
    # forward, timed
    u.zero_()
    v.copy_(v0t)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = g.step(u, v, None, nsteps=nsteps, dt=dt, v_prescribed=vpt)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    res.update({"forward_s": round(t_fwd, 4), "steps_per_s": round(nsteps / t_fwd, 1),
                "dof_steps_per_s": 2 * w.N * nsteps / t_fwd, "bonds_broken": st.newly_broken,
                "u_final_l2": float(torch.linalg.norm(u))})
    # forward + checkpointed adjoint, timed
    g.set_bond_mask(mask0)
    E = Et.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    uN = verlet_run(g, E, torch.zeros_like(u), v0t.clone(), nsteps, dt, v_prescribed=vpt, checkpoint_every=45)
    loss = 0.5 * (uN * uN).sum()
    loss.backward()
    torch.cuda.synchronize()
    res.update({"forward_plus_adjoint_s": round(time.perf_counter() - t0, 4), "loss": float(loss.detach()),
                "grad_E_l2": float(torch.linalg.norm(E.grad)), "checkpoint_every": 45})
    # the first 100 steps against the oracle's Verlet loop from the same state
    g.set_bond_mask(mask0)
    u.zero_()
    v.copy_(v0t)
    st = g.step(u, v, None, nsteps=100, dt=dt, v_prescribed=vpt)
    mu = oracle.intact_mu(2, w.n, w.M)
    oracle.prenotch(w.n, w.M, w.extra["notch"], w.extra["notch_den"], mu)
    uo, vo = np.zeros((2,) + lay.shape), v_init.copy()
    nb = oracle.vv(2, w.n, w.h, w.M, oracle.alpha(2, 1.0, w.delta), uo, vo, 100, dt, E=E_np, mu=mu, s0=w.s0,
                   cons=cons, vpres=vp)
    res["first_100_steps_vs_oracle"] = {"u_rel_l2": _rel(u.cpu().numpy(), uo), "v_rel_l2": _rel(v.cpu().numpy(), vo),
                                        "bonds_broken_gpu": st.newly_broken, "bonds_broken_oracle": nb}
    g.close()
    return res


def _extras(torch, pd, syn, dev):
    """Secondary measurements (rank 0): variants, CG, cube, crack loop; every
    result with its error against the FP64 oracle (computed after timing)."""
    import numpy as np
    import oracle
    out = {}
    # measured arithmetic peaks (the denominators of the ALU-bound kernels)
    peaks = {"fp32_tflops": pd.pd_probe_fma_rate(pd.PD_F32) / 1e12, "fp64_tflops": pd.pd_probe_fma_rate(pd.PD_F64) / 1e12}
    out["alu_peaks_measured"] = {k: round(v, 2) for k, v in peaks.items()}
    variants, verr, vfrac, vfrac32 = {}, {}, {}, {}
    for M in (3, 6):
        w = syn.large_plate(M)
        g = pd.Grid(2, w.n, w.h, w.M)
        al = oracle.alpha(2, 1.0, w.delta)
        for dt, name in ((torch.float32, "f32"), (torch.float64, "f64")):
            B = 8 if dt == torch.float32 else 4
            U = torch.rand((B, 2, NSIDE, NSIDE), dtype=dt, device=dev) * 2 - 1
            O = torch.empty_like(U)
            ref0 = oracle.stiffness(2, w.n, w.h, w.M, al, U[0].double().cpu().numpy())
            # FP64 "stencil": the pair form on u minus each tile's plane (the default);
            # "stencil_difference": the difference form; "stencil_pair": the pair form on u
            for meth, mname in ((pd.PD_METHOD_STENCIL, "stencil"), (pd.PD_METHOD_STENCIL | pd.PD_PAIR_FORM, "stencil_pair"),
                                (pd.PD_METHOD_STENCIL | pd.PD_ACCURATE, "stencil_difference"),
                                (pd.PD_METHOD_STENCIL | pd.PD_NO_TMA, "stencil_plain"), (pd.PD_METHOD_FFT, "fft")):
                if (name == "f64" and mname == "stencil_plain") or (name == "f32" and mname == "stencil_difference"):
                    continue
                key = f"M{M}_{name}_{mname}"
                try:
                    t = _time_fn(torch, lambda: g.matvec(U, O, flags=meth), reps=10)
                    variants[key] = round(B * 2 * w.N / t / 1e9, 2)
                    g.matvec(U, O, flags=meth)
                    torch.cuda.synchronize()
                    verr[key] = _rel(O[0].double().cpu().numpy(), ref0)
                except pd.PDError:
                    variants[key] = None
            del U, O
        # FP64 stencil: FLOPs of the pair form per output (general pair 10, axis pair 3, diagonal 8)
        npairs = oracle.offsets(2, M).shape[0] // 2
        gen = npairs - 2 * M
        f64_flops = (gen * 10 + 2 * M * 3 + 8) * w.N
        for key in (f"M{M}_f64_stencil", f"M{M}_f64_stencil_pair", f"M{M}_f64_stencil_difference"):
            if variants.get(key):
                vfrac[key] = round(variants[key] * 1e9 / 2 * (f64_flops / w.N) / (peaks["fp64_tflops"] * 1e12), 3)
        # FP32 stencils against the measured FP32 FMA rate with the same algorithmic FLOP count:
        # beyond M = 3 the FP32 product is bound by the FMA pipe, not by HBM
        for key in (f"M{M}_f32_stencil", f"M{M}_f32_stencil_pair"):
            if variants.get(key):
                vfrac32[key] = round(variants[key] * 1e9 / 2 * (f64_flops / w.N) / (peaks["fp32_tflops"] * 1e12), 3)
        g.close()
    out["variants_gdofs"] = variants
    out["variants_rel_l2_vs_oracle"] = {k: float(f"{v:.3e}") for k, v in verr.items()}
    out["variants_fp64_frac_of_measured_fp64_peak"] = vfrac
    out["variants_fp32_frac_of_measured_fp32_peak"] = vfrac32
    out["cufft_comparison"] = _cufft_comparison(torch, pd, syn, dev, oracle)
    # the autotuner's choice (method; FP32 2D stencil tile height) per horizon and precision on
    # the 1024^2 plate and the 128^3 cube, with the time of each candidate; "fixed" is the
    # 64 x 32 stencil tile
    tune = {}
    for key, w in (("plate1024_M3", syn.large_plate(3)), ("plate1024_M4", syn.large_plate(4)),
                   ("plate1024_M6", syn.large_plate(6)), ("cube128_M3", syn.cube(128, 3))):
        g = pd.Grid(w.dim, w.n, w.h, w.M)
        t = g.autotune()
        info = pd.pd_get_info(g.handle)
        ent = {k: round(v, 4) for k, v in t.items()}
        ent["f32_method"] = "fft" if info.auto_method[0] == pd.PD_METHOD_FFT else "stencil"
        ent["f64_method"] = "fft" if info.auto_method[1] == pd.PD_METHOD_FFT else "stencil"
        ent["f32_stencil_tile_rows"] = int(info.stencil_tile_rows)
        if w.dim == 2 and w.M <= 4:
            g.set_stencil_tile_rows(32)
            U = torch.zeros((1, 2) + tuple(reversed(w.n)), dtype=torch.float32, device=dev)
            O = torch.empty_like(U)
            ent["f32_stencil_fixed_tile32_ms"] = round(_time_fn(torch, lambda: g.matvec(U, O, flags=pd.PD_METHOD_STENCIL),
                                                                reps=20) * 1e3, 4)
            g.set_stencil_tile_rows(ent["f32_stencil_tile_rows"])
        tune[key] = ent
        g.close()
    out["autotune_ms_per_field"] = tune
    # static solve on the 1024^2 plate (clamp left, traction right), rtol 1e-8
    w = syn.large_plate(3)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    g.autotune()
    b = torch.tensor(w.b, device=dev)
    cg = {}
    for mode, name in ((pd.PD_CG_MIXED, "mixed"), (pd.PD_CG_F64, "f64")):
        u = torch.zeros_like(b)
        pd.pd_cg_solve(g.handle, b, u, 1e-8, 64, mode, allow_not_converged=True)   # warm: workspace, graphs
        u.zero_()
        torch.cuda.synchronize()
        st = pd.pd_cg_solve(g.handle, b, u, 1e-8, 400000, mode, allow_not_converged=True)
        cg[name] = {"seconds": round(st.seconds, 4), "iterations": st.iterations, "outer": st.outer,
                    "f64_matvecs": st.f64_matvecs, "rel_residual": st.rel_residual,
                    "true_rel_residual_oracle": _true_residual(oracle, 2, w, u.cpu().numpy(), w.b, w.constrained,
                                                               oracle.alpha(2, 1.0, w.delta))}
    if cg["mixed"]["seconds"] > 0:
        cg["speedup_mixed_vs_f64"] = round(cg["f64"]["seconds"] / cg["mixed"]["seconds"], 3)
    out["cg_1024_rtol1e-8"] = cg
    # the paper's static solver (ADR/CDEI, Algorithm 1) on the same plate and rtol: FP64, and FP32
    # operator with FP64 refresh
    adr1024 = {}
    for mode, name in ((pd.PD_ADR_F64, "f64"), (pd.PD_ADR_MIXED, "mixed")):
        u = torch.zeros_like(b)
        pd.pd_adr_solve(g.handle, b, u, 1e-8, 64, allow_not_converged=True, mode=mode)   # warm: workspace, graph
        u.zero_()
        torch.cuda.synchronize()
        st = pd.pd_adr_solve(g.handle, b, u, 1e-8, 1_000_000, allow_not_converged=True, mode=mode)
        adr1024[name] = {"seconds": round(st.seconds, 4), "iterations": st.iterations, "outer": st.outer,
                         "rel_residual": st.rel_residual,
                         "us_per_iteration": round(st.seconds / max(1, st.iterations) * 1e6, 2),
                         "true_rel_residual_oracle": _true_residual(oracle, 2, w, u.cpu().numpy(), w.b,
                                                                    w.constrained, oracle.alpha(2, 1.0, w.delta))}
    adr1024["speedup_mixed_vs_f64"] = round(adr1024["f64"]["seconds"] / adr1024["mixed"]["seconds"], 3)
    out["adr_1024_rtol1e-8"] = adr1024
    g.close()
    # ADR for the step counts of the paper's 2D static runs (plate meshes 400x200 .. 1600x800)
    adr = {}
    for nx, ny, steps in ((400, 200, 3000), (800, 400, 4000), (1600, 800, 5000)):
        n = (nx, ny)
        cons = syn.clamp_left(2, n, 3)
        bb = torch.tensor(syn.traction_right(2, n, 3, 1e-3), device=dev)
        g = pd.Grid(2, n, 1.0 / nx, 3, constrained=cons)
        u = torch.zeros_like(bb)
        pd.pd_adr_solve(g.handle, bb, u, 1e-30, 64, allow_not_converged=True)
        u.zero_()
        torch.cuda.synchronize()
        st = pd.pd_adr_solve(g.handle, bb, u, 1e-30, steps, allow_not_converged=True)
        u.zero_()
        pd.pd_adr_solve(g.handle, bb, u, 1e-30, 64, allow_not_converged=True, mode=pd.PD_ADR_MIXED)
        u.zero_()
        torch.cuda.synchronize()
        stm = pd.pd_adr_solve(g.handle, bb, u, 1e-30, steps, allow_not_converged=True, mode=pd.PD_ADR_MIXED)
        adr[f"{nx}x{ny}"] = {"steps": st.iterations, "seconds": round(st.seconds, 4),
                             "dof_steps_per_s": 2 * nx * ny * st.iterations / st.seconds,
                             "mixed_seconds": round(stm.seconds, 4)}
        g.close()
    out["adr_plate_fixed_steps"] = adr
    # surface correction (volume method): its cost on the timed FP32 product, and ADR with it
    w = syn.large_plate(3)
    g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
    U = torch.rand((8, 2, NSIDE, NSIDE), dtype=torch.float32, device=dev) * 2 - 1
    O = torch.empty_like(U)
    fl = pd.PD_METHOD_STENCIL | pd.PD_PROJECT
    t0_ = _time_fn(torch, lambda: g.matvec(U, O, flags=fl), reps=10)
    g.set_surface_correction(pd.PD_SC_VOLUME)
    t1_ = _time_fn(torch, lambda: g.matvec(U, O, flags=fl), reps=10)
    sc = {"f32_stencil_gdofs": round(8 * 2 * w.N / t0_ / 1e9, 2),
          "f32_stencil_with_correction_gdofs": round(8 * 2 * w.N / t1_ / 1e9, 2),
          "correction_us_per_field": round((t1_ - t0_) / 8 * 1e6, 2)}
    del U, O
    g.close()
    for nx, ny, steps in ((400, 200, 3000), (800, 400, 4000), (1600, 800, 5000)):
        n = (nx, ny)
        bb = torch.tensor(syn.traction_right(2, n, 3, 1e-3), device=dev)
        g = pd.Grid(2, n, 1.0 / nx, 3, constrained=syn.clamp_left(2, n, 3), surface_correction=pd.PD_SC_VOLUME)
        u = torch.zeros_like(bb)
        pd.pd_adr_solve(g.handle, bb, u, 1e-30, 64, allow_not_converged=True)
        u.zero_()
        torch.cuda.synchronize()
        st = pd.pd_adr_solve(g.handle, bb, u, 1e-30, steps, allow_not_converged=True)
        sc[f"adr_{nx}x{ny}_{steps}_steps_s"] = round(st.seconds, 4)
        g.close()
    out["surface_correction"] = sc
    # 64 uneven plates (sides 128..512, M in {3,4}): one batched solve vs one solve per plate
    plates = syn.batched_plates(64)
    grids = [pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained) for w in plates]
    bs = [torch.tensor(w.b, device=dev) for w in plates]
    dof = sum(2 * w.N for w in plates)
    bt = pd.pd_batch_create(grids)
    us = [torch.zeros_like(x) for x in bs]
    pd.pd_batch_cg_solve(bt, bs, us, 1e-8, 64, allow_not_converged=True)   # warm: graph capture
    for u in us:
        u.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = pd.pd_batch_cg_solve(bt, bs, us, 1e-8, 1_000_000)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    pd.pd_batch_destroy(bt)
    batch_true = max(_true_residual(oracle, 2, wp, up.cpu().numpy(), wp.b, wp.constrained,
                                    oracle.alpha(2, 1.0, wp.delta)) for wp, up in zip(plates, us))
    for g_, b_ in zip(grids, bs):   # warm each plate's own workspace and graphs
        pd.pd_cg_solve(g_.handle, b_, torch.zeros_like(b_), 1e-8, 64, pd.PD_CG_MIXED, allow_not_converged=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g_, b_ in zip(grids, bs):
        pd.pd_cg_solve(g_.handle, b_, torch.zeros_like(b_), 1e-8, 1_000_000, pd.PD_CG_MIXED)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    out["batch_64_plates_rtol1e-8"] = {
        "dof_total": dof, "batched_s": round(t_batch, 4), "sequential_s": round(t_seq, 4),
        "batched_dof_per_s": dof / t_batch, "sequential_dof_per_s": dof / t_seq,
        "speedup": round(t_seq / t_batch, 3), "max_rel_residual": max(s.rel_residual for s in st),
        "max_true_rel_residual_oracle": batch_true,
        "max_inner_iterations": max(s.iterations for s in st)}
    for g_ in grids:
        g_.close()
    # 3D cube 128^3, FP32
    w = syn.cube(128, 3)
    g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained)
    cube = {}
    for dt_, name in ((torch.float32, "f32"), (torch.float64, "f64")):
        U = torch.tensor(w.u, dtype=dt_, device=dev)
        O = torch.empty_like(U)
        for meth, mname in ((pd.PD_METHOD_STENCIL, "stencil"), (pd.PD_METHOD_FFT, "fft")):
            s = _time_fn(torch, lambda: g.matvec(U, O, flags=meth | pd.PD_PROJECT), reps=10)
            cube[f"{name}_{mname}_gdofs"] = round(3 * w.N / s / 1e9, 2)
    # every product against the FP64 oracle on the same (rounded) input
    al3 = oracle.alpha(3, 1.0, w.delta)
    for dt_, name in ((torch.float32, "f32"), (torch.float64, "f64")):
        U = torch.tensor(w.u, dtype=dt_, device=dev)
        ref = oracle.stiffness(3, w.n, w.h, w.M, al3, U.double().cpu().numpy(), cons=w.constrained)
        for meth, mname in ((pd.PD_METHOD_STENCIL, "stencil"), (pd.PD_METHOD_FFT, "fft")):
            o = g.matvec(U, flags=meth | pd.PD_PROJECT).double().cpu().numpy()
            cube[f"{name}_{mname}_rel_l2_vs_oracle"] = _rel(o, ref)
    del U
    g.autotune()
    b = torch.tensor(w.b, device=dev)
    for mode, name in ((pd.PD_CG_MIXED, "cg_mixed"), (pd.PD_CG_F64, "cg_f64")):
        u = torch.zeros_like(b)
        pd.pd_cg_solve(g.handle, b, u, 1e-8, 32, mode, allow_not_converged=True)
        u.zero_()
        st = pd.pd_cg_solve(g.handle, b, u, 1e-8, 200000, mode, allow_not_converged=True)
        cube[name] = {"seconds": round(st.seconds, 4), "iterations": st.iterations, "rel_residual": st.rel_residual,
                      "true_rel_residual_oracle": _true_residual(oracle, 3, w, u.cpu().numpy(), w.b, w.constrained,
                                                                 al3)}
    out["cube128"] = cube
    g.close()
    out["crack512"] = _crack512(torch, pd, syn, dev, oracle)
    # 3D block with two through-thickness notches (the Kalthoff-Winkler geometry of Sec. 5.4,
    # the impactor replaced by a velocity zone): the paper's 1350 steps on its coarse mesh,
    # 200 steps on its fine one
    kw = {}
    for nx, ny, nz, steps in ((201, 101, 9, 1350), (402, 202, 18, 200)):
        w = syn.kw_block(nx, ny, nz, 3)
        g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained, s0=w.s0)
        notch_bonds = sum(g.break_segment(seg, w.extra["notch_den"]) for seg in w.extra["notches"])
        vpt = torch.tensor(w.extra["v_prescribed"], device=dev)
        u = torch.zeros_like(vpt)
        v = vpt.clone()
        dt_kw = w.extra["dt"]
        g.step(u, v, None, nsteps=5, dt=dt_kw, v_prescribed=vpt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = g.step(u, v, None, nsteps=steps, dt=dt_kw, v_prescribed=vpt)
        torch.cuda.synchronize()
        t_kw = time.perf_counter() - t0
        kw[f"{nx}x{ny}x{nz}"] = {"steps": steps, "seconds": round(t_kw, 4), "steps_per_s": round(steps / t_kw, 1),
                                 "dof_steps_per_s": 3 * w.N * steps / t_kw, "notch_bonds": notch_bonds,
                                 "bonds_broken_in_run": st.newly_broken}
        g.close()
    out["kw3d_verlet"] = kw
    return out


CASES = ("fft2d", "fft2d_f64", "stencil2d_f64", "walk2d", "stencil3d", "fft3d", "crack", "cg", "adr", "adr_mixed", "sc", "kw3d")


def run_case(args):
    """One secondary workload in a loop (for ncu launch lists and captures); prints one JSON line.

    fft2d: K u, 1024^2 plate, M=3, FP32 FFT tiles, 8 fields.  stencil2d_f64: the same with the FP64
    stencil, 4 fields.  walk2d: the same with the FP32 column walk, 16 fields.  fft2d_f64: FP64 FFT
    tiles at M=6, 2 fields.  stencil3d / fft3d: K u on the 128^3 cube, M=3, FP32.  crack: one Verlet step
    with bond breaking on the pre-notched 512^2 plate.  cg: 64 iterations of the mixed CG on the
    1024^2 plate (graph-replayed inner loop).  adr / adr_mixed: 64 ADR iterations (Algorithm 1, FP64 /
    mixed) on that plate.  sc: K u with the surface correction, 1024^2, FP32, 8 fields.  kw3d: one Verlet
    step on the notched 201x101x9 block."""
    import numpy as np
    import torch
    import paper_2301_11828_gb300 as pd
    import synthetic as syn
    pd.load_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    case = args.case
    if case in ("fft2d", "fft2d_f64", "stencil2d_f64", "walk2d"):
        w = syn.large_plate(6 if case == "fft2d_f64" else 3)
        g = pd.Grid(2, w.n, w.h, w.M)
        dt, B, meth = {"fft2d": (torch.float32, 8, pd.PD_METHOD_FFT),
                       "fft2d_f64": (torch.float64, 2, pd.PD_METHOD_FFT),
                       "stencil2d_f64": (torch.float64, 4, pd.PD_METHOD_STENCIL),
                       "walk2d": (torch.float32, 16, pd.PD_METHOD_STENCIL)}[case]
        if case == "walk2d":
            g.set_stencil_tile_rows(0)   # the column walk
        U = torch.rand((B, 2, NSIDE, NSIDE), dtype=dt, device=dev) * 2 - 1
        O = torch.empty_like(U)
        step, units = (lambda: g.matvec(U, O, flags=meth)), B * 2 * w.N
    elif case in ("stencil3d", "fft3d"):
        w = syn.cube(128, 3)
        g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained)
        U = torch.tensor(w.u, dtype=torch.float32, device=dev)
        O = torch.empty_like(U)
        meth = pd.PD_METHOD_STENCIL if case == "stencil3d" else pd.PD_METHOD_FFT
        step, units = (lambda: g.matvec(U, O, flags=meth | pd.PD_PROJECT)), 3 * w.N
    elif case == "crack":
        w = syn.crack_plate(512, 3)
        lay = w.extra["vel_layers"]
        cons = np.zeros((2,) + lay.shape, dtype=np.uint8)
        cons[1] = lay != 0
        vp = np.zeros((2,) + lay.shape)
        vp[1] = lay * w.extra["v0"]
        g = pd.Grid(2, w.n, w.h, w.M, constrained=cons, E_field=torch.tensor(w.extra["E_field"], device=dev), s0=w.s0)
        g.break_segment(w.extra["notch"], w.extra["notch_den"])
        vpt = torch.tensor(vp, device=dev)
        u = torch.zeros((2,) + lay.shape, dtype=torch.float64, device=dev)
        v = vpt.clone()
        step, units = (lambda: g.step(u, v, None, nsteps=1, dt=2.99e-3, v_prescribed=vpt)), 2 * w.N
    elif case in ("adr", "adr_mixed"):
        w = syn.large_plate(3)
        g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
        b = torch.tensor(w.b, device=dev)
        u = torch.zeros_like(b)
        mode = pd.PD_ADR_F64 if case == "adr" else pd.PD_ADR_MIXED

        def step():
            u.zero_()
            pd.pd_adr_solve(g.handle, b, u, 1e-30, 64, allow_not_converged=True, mode=mode)
        units = 64
    elif case == "sc":
        w = syn.large_plate(3)
        g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained, surface_correction=pd.PD_SC_VOLUME)
        U = torch.rand((8, 2, NSIDE, NSIDE), dtype=torch.float32, device=dev) * 2 - 1
        O = torch.empty_like(U)
        step, units = (lambda: g.matvec(U, O, flags=pd.PD_METHOD_STENCIL)), 8 * 2 * w.N
    elif case == "kw3d":
        w = syn.kw_block(201, 101, 9, 3)
        g = pd.Grid(3, w.n, w.h, w.M, constrained=w.constrained, s0=w.s0)
        for seg in w.extra["notches"]:
            g.break_segment(seg, w.extra["notch_den"])
        vpt = torch.tensor(w.extra["v_prescribed"], device=dev)
        u = torch.zeros_like(vpt)
        v = vpt.clone()
        step, units = (lambda: g.step(u, v, None, nsteps=1, dt=w.extra["dt"], v_prescribed=vpt)), 3 * w.N
    elif case == "cg":
        w = syn.large_plate(3)
        g = pd.Grid(2, w.n, w.h, w.M, constrained=w.constrained)
        b = torch.tensor(w.b, device=dev)
        u = torch.zeros_like(b)

        def step():
            u.zero_()
            pd.pd_cg_solve(g.handle, b, u, 1e-30, 64, pd.PD_CG_MIXED, allow_not_converged=True)
        units = 64
    else:
        raise SystemExit(f"unknown case {case}")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    dt_s = (time.perf_counter() - t0) / args.steps
    print(json.dumps({"case": case, "steps": args.steps, "ms_per_step": dt_s * 1e3,
                      "units_per_step": units, "units_per_s": units / dt_s}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--quick", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle check of the timed outputs")
    ap.add_argument("--case", choices=CASES, default=None,
                    help="run one secondary workload in a loop instead of the headline (profiling)")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
