#!/usr/bin/env python
"""Throughput of the fused pseudopotential D2Q9 step (MLUPS and HBM roofline).

Workload (one "step" = one lattice Boltzmann time step of the whole domain):
8192 x 8192 periodic D2Q9, spinodal decomposition from
rho = rho_avg (1 + 0.01 U[-1, 1]) (seed 3 + rank) with rho_avg midway between
the Maxwell coexistence densities at T = 0.85 Tc, tau = 0.8, improved forcing
scheme with sigma = 0.1, FP32 populations.  The populations (2 x 2.4 GB)
are far larger than L2, so no flush is needed between steps.

* value      -- MLUPS over all ranks, device time of exactly K steps (CUDA
                events on the stream the kernels run on), inputs resident.
* roofline   -- the step kernel: algorithmic bytes per launch (9 reads + 9
                writes per cell) / average launch time, against the measured
                HBM copy bandwidth.
* e2e        -- the same metric through the public C ABI from page-locked
                host buffers (lbm_host_alloc): lbm_init_density (H2D), K
                steps, lbm_get_moments (D2H); median of three passes.
* cpu_baseline -- the FP64 oracle (test infrastructure) on a bounded sample
                of the same workload, on this host's cores.
* storage_variants, schemes_fp32 (every forcing scheme and the MRT form on
  the same workload), batched_sweep (128 slabs, with the sequential plain runs
  measured over all of them), batched_sweep_config4_512 (the 512-slab sweep,
  batched), warm_start (a reduced config 5) -- the other workloads' legs.

``--impl reference`` times the oracle alone as the reference arm.
Under torchrun every rank runs its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 pseudopotential MLUPS & % HBM roofline; batched sweep; warm-start speedup"
BYTES_PER_CELL = {"fp32": 72, "fp64": 144, "bf16dev": 44, "fp16dev": 44}
KERNEL_SOURCES = ["lbm_device.cuh", "lbm_kernels.cuh", "lbm_launch.cuh"]
STORE_NAMES = {"fp32": "StoreF32", "fp64": "StoreF64", "bf16dev": "StoreBF16",
               "fp16dev": "StoreF16"}
# DRAM bytes per launch of the step kernel from an ncu capture, keyed by the
# hash of the kernel sources it was taken on (null once they change), the
# storage type, the lattice side and the kernel variant.  Captures of the
# whole 8192^2 workload take only timing; DRAM counters come from a 4096^2
# capture of the same kernel, scaled by the cell count.
MEASURED_TRAFFIC = {
    # ncu launch list, 25 launches of strip_kernel<StoreF32, improved, step> at
    # 8192^2: 2.437 GB read + 2.370 GB written per launch
    ("8a40f73e27882b9d", "fp32", 8192, "register"): 4.807e9,
    # ncu launch list, 25 launches of strip2_kernel<StoreF32, improved, step>
    # at 8192^2: 2.431 GB read + 2.368 GB written per launch
    ("c8b20c715c92ee44", "fp32", 8192, "pair"): 4.7996e9,
    # the same after the fetch / assemble split of the row loads (4 CTAs/SM):
    # 2.431 GB read + 2.368 GB written per launch
    ("a776dde1b00b0c71", "fp32", 8192, "pair"): 4.7986e9,
    # the same kernel after comment edits and packed 16-bit conversions
    # (FP32 code unchanged): 2.431 GB read + 2.368 GB written per launch
    ("187a00600d401039", "fp32", 8192, "pair"): 4.7984e9,
    # after adding the MRT scheme (three rates in the kernel arguments):
    # 2.431 GB read + 2.368 GB written per launch
    ("7bc3668251e0d237", "fp32", 8192, "pair"): 4.7986e9,
    # packed FP32x2 pair arithmetic, row range of a band: small-case capture
    # (-k strip2_kernel -c 3 at 4096^2: 615.3 MB read + 555.5 MB written per
    # launch on average), scaled to 8192^2 by the cell count (x 4)
    ("ee1858b957fb85d9", "fp32", 8192, "pair"): 4.6832e9,
    # the same kernel source after the padded-pitch template parameter of the
    # batch body (single lattices unpadded): 4096^2 capture 615.3 MB read +
    # 555.6 MB written per launch, x4 cells
    ("8f05beea9b05b658", "fp32", 8192, "pair"): 4.6838e9,
    # after the band prologue fetched its three rows together: 4096^2 capture
    # 615.3 MB read + 555.6 MB written per launch, x4 cells
    ("300215b053bb1d0a", "fp32", 8192, "pair"): 4.6836e9,
    # rows fetched into shared memory with cp.async: 4096^2 capture 616.7 MB
    # read + 555.6 MB written per launch, x4 cells
    ("1026352877ad7d4b", "fp32", 8192, "pair"): 4.6892e9,
    # the same FP32 kernel after the 16-bit unpack change (StoreBF16 only):
    # 4096^2 capture 616.8 MB read + 555.5 MB written per launch, x4 cells
    ("01946c2627dbfadb", "fp32", 8192, "pair"): 4.6893e9,
    # after the odd-nx store change of the batch body (single lattices
    # unpadded) and narrower compiler barriers around the row copies: 4096^2
    # capture 616.7 MB read + 555.8 MB written per launch, x4 cells
    ("93fd099c0bd56bf9", "fp32", 8192, "pair"): 4.6899e9,
    # buffer pointers held in registers on the row-copy path, copy stores
    # addressed from the pair store: 4096^2 capture 616.7 MB read + 555.8 MB
    # written per launch, x4 cells
    ("078d563a4c56ea55", "fp32", 8192, "pair"): 4.6899e9,
    # the same FP32 kernel after the 16-bit decode / residual change (16-bit
    # paths only): 4096^2 capture 616.8 MB read + 555.9 MB written, x4 cells
    ("bab0aef77fdf5a50", "fp32", 8192, "pair"): 4.6906e9,
    # keys from here on hash the kernels' code without comments (the same
    # capture as the entry above: 616.8 MB read + 555.9 MB written at 4096^2)
    ("cac15c6501ae37f0", "fp32", 8192, "pair"): 4.6906e9,
}


def kernel_source_hash():
    """Hash of the step kernels' code: the kernel sources with their comments
    and blank lines removed, so that a comment edit keeps the traffic
    counters taken for the code, and any code change drops them."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1204_4098_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)  # block comments
        for line in text.splitlines():
            code = re.sub(r"//.*$", "", line).rstrip()
            if code.strip():
                h.update((code + "\n").encode())
    return "c" + h.hexdigest()[:15]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "100", "-f", self.path]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_density(n, rank, T_over_Tc=0.85):
    from paper_1204_4098_gb300 import inputs, lbm
    rg, rl, _ = lbm.maxwell(lbm.temperature(T_over_Tc))
    return inputs.spinodal(n, n, 0.5 * (rg + rl), amp=0.01, seed=3 + rank), (rg, rl)


def host_description():
    """Host CPU of this machine: model name and the cores this process may use."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip() and v.strip() != "-":
                model = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"cpu_model": model, "nproc": usable, "machine": os.uname().machine}


def _time_oracle(lib, nx, ny, steps, init, scheme, tau, sigma, t):
    import oracle
    lat = oracle.Lattice(nx, ny, t, lib=lib)
    lat.init_density(init)
    t0 = time.perf_counter()
    rc, done = lat.step(steps, scheme, tau, sigma)
    dt = time.perf_counter() - t0
    assert rc == 0
    return nx * ny * done / dt / 1e6, dt, done


def cpu_baseline(n_side=1024, steps_1=40, steps_all=200, config1_steps=10000):
    """FP64 oracle (test infrastructure) on the host cores: the 1024 x 1024
    sample of the workload recipe (improved sigma = 0.1, T = 0.85 Tc,
    tau = 0.8, spinodal init seed 3) on one core and on all cores (the
    oracle's OpenMP build, bit-identical), and the 64 x 64 flat-interface
    slab (Shan-Chen, tau = 1, T = 0.8 Tc, 1e4 steps) likewise.  The headline
    value is the all-core sample."""
    import oracle
    from oracle import theory as th
    from paper_1204_4098_gb300 import inputs
    host = host_description()
    t = 0.85
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(t)))
    rho0 = inputs.spinodal(n_side, n_side, 0.5 * (rg + rl), amp=0.01, seed=3)
    one = oracle.load()
    omp, threads = oracle.load_omp(host["nproc"])
    v1, dt1, d1 = _time_oracle(one, n_side, n_side, steps_1, rho0, oracle.IMPROVED, 0.8, 0.1, t)
    out = {"unit": "MLUPS", "kind": "oracle", "host": host,
           "single_core": {"value": v1, "cores": 1,
                           "sample": f"{n_side}x{n_side} crop, {d1} steps, 1 thread "
                                     f"({dt1:.1f} s)"}}
    if omp is not None:
        va, dta, da = _time_oracle(omp, n_side, n_side, steps_all, rho0, oracle.IMPROVED, 0.8,
                                   0.1, t)
        out.update({"value": va, "cores": threads,
                    "sample": f"{n_side}x{n_side} crop of the workload recipe, {da} steps, FP64, "
                              f"{threads} threads (OpenMP build, bit-identical; {dta:.1f} s)"})
    else:
        out.update({"value": v1, "cores": 1, "sample": out["single_core"]["sample"]})
    # config 1 in full: 64 x 64 slab at the Maxwell densities, 1e4 steps
    t1 = 0.8
    g1, l1, _ = th.maxwell(th.CarnahanStarling(th.temperature(t1)))
    slab = inputs.slab_step(64, 64, g1, l1, 16, 48, amp=1e-3, seed=1)
    c1 = {}
    for name, lib, cores in (("single_core", one, 1), ("all_cores", omp, threads)):
        if lib is None:
            continue
        v, dt, d = _time_oracle(lib, 64, 64, config1_steps, slab, oracle.SC, 1.0, 0.0, t1)
        c1[name] = {"value": v, "cores": cores, "seconds": dt, "steps": d}
    out["config1_64x64_1e4_steps"] = c1
    return out


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle
    from oracle import theory as th
    from paper_1204_4098_gb300 import inputs
    side = args.ref_side
    t = 0.85
    host = host_description()
    lib, threads = oracle.load_omp(host["nproc"])
    if lib is None:
        lib, threads = oracle.load(), 1
    rg, rl, _ = th.maxwell(th.CarnahanStarling(th.temperature(t)))
    lat = oracle.Lattice(side, side, t, lib=lib)
    lat.init_density(inputs.spinodal(side, side, 0.5 * (rg + rl), amp=0.01, seed=3))
    lat.step(args.warmup, oracle.IMPROVED, 0.8, 0.1)
    t0 = time.perf_counter()
    rc, done = lat.step(args.steps, oracle.IMPROVED, 0.8, 0.1)
    dt = time.perf_counter() - t0
    value = side * side * done / dt / 1e6
    sample = (f"{side}x{side} crop of the 8192x8192 recipe per step, FP64 oracle, "
              f"{threads} threads (OpenMP build)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / max(done, 1) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": sample, "host": host},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": f"{args.n}x{args.n} periodic D2Q9 spinodal decomposition, "
                        f"T=0.85Tc, tau=0.8, improved forcing sigma=0.1, "
                        f"{args.precision} populations",
            "nx": args.n, "ny": args.n, "scheme": "improved", "sigma": 0.1, "tau": 0.8,
            "T_over_Tc": 0.85, "precision": args.precision,
            "l2": "inputs larger than L2 (two population buffers of "
                  f"{args.n * args.n * BYTES_PER_CELL[args.precision] / 2 / 1e9:.1f} GB each)"}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1204_4098_gb300 import lbm

    torch.cuda.set_device(local)
    # a dedicated stream: the library runs on it and the events are recorded on it
    stream = torch.cuda.Stream(device=local)
    assert stream.cuda_stream != 0
    prec = {"fp32": lbm.FP32, "fp64": lbm.FP64, "bf16dev": lbm.BF16DEV,
            "fp16dev": lbm.FP16DEV}[args.precision]
    n = args.n
    rho0, _ = workload_density(n, rank)
    cells = n * n

    lat = lbm.Lattice(n, n, 0.85, precision=prec, device=local, stream=stream.cuda_stream)
    lat.set_variant({"auto": lbm.VARIANT_AUTO, "register": lbm.VARIANT_REGISTER,
                     "pair": lbm.VARIANT_PAIR, "staged": lbm.VARIANT_STAGED}[args.kernel_variant])
    lat.init_density(rho0)
    lat.step_async(args.warmup, lbm.IMPROVED, 0.8, 0.1)
    assert lat.sync() == lbm.LBM_OK

    props = torch.cuda.get_device_properties(local)
    bus = None
    if hasattr(props, "pci_bus_id"):
        bus = f"{getattr(props, 'pci_domain_id', 0):08X}:{props.pci_bus_id:02X}:" \
              f"{getattr(props, 'pci_device_id', 0):02X}.0"
    sampler = ClockSampler(bus)
    sampler.start()

    # ---- device-resident timing: exactly K steps, one kernel launch each ----
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist_barrier(world)
    torch.cuda.synchronize()
    launches0 = lbm.launch_count()
    start.record(stream)
    lat.step_async(args.steps, lbm.IMPROVED, 0.8, 0.1)
    end.record(stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    launches = lbm.launch_count() - launches0
    variant_used = lat.variant()
    ms = start.elapsed_time(end)
    assert lat.sync() == lbm.LBM_OK
    clocks = sampler.stop()
    ms_max = dist_max(ms, world)
    value = world * cells * args.steps / (ms_max * 1e-3) / 1e6

    per_launch_s = ms * 1e-3 / args.steps
    bpc = BYTES_PER_CELL[args.precision]
    achieved = bpc * cells / per_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    vname = {lbm.VARIANT_REGISTER: "register", lbm.VARIANT_PAIR: "pair",
             lbm.VARIANT_STAGED: "staged"}.get(variant_used, "register")
    traffic = MEASURED_TRAFFIC.get((kernel_source_hash(), args.precision, n, vname))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": {lbm.VARIANT_PAIR: "strip2_kernel", lbm.VARIANT_STAGED:
                           "strip_tma_kernel"}.get(variant_used, "strip_kernel")
                + f"<{STORE_NAMES[args.precision]}, improved, step>",
                "algorithmic_bytes_per_launch": bpc * cells,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s"}

    # ---- end to end through the C ABI with page-locked host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = lambda: lbm.host_array((n, n))  # page-locked, huge pages where available
        h_rho0 = pin()
        h_rho0[...] = rho0
        outs = (pin(), pin(), pin())
        # one untimed pass through the same calls first (warm-up, like the
        # device-timed steps): the page-locked buffers' first transfers
        lat.init_density(h_rho0)
        lat.step_async(1, lbm.IMPROVED, 0.8, 0.1)
        lat.observe(out=outs)
        # three timed passes, the median reported: the host copies share the
        # host's memory with whatever else runs there
        samples = []
        for _ in range(3):
            dist_barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.init_density(h_rho0)
            lat.step_async(args.steps, lbm.IMPROVED, 0.8, 0.1)
            lat.observe(out=outs)
            torch.cuda.synchronize()
            dt = dist_max(time.perf_counter() - t0, world)
            assert np.isfinite(outs[0][0, 0])
            samples.append(world * cells * args.steps / dt / 1e6)
        e2e = {"value": float(np.median(samples)), "unit": "MLUPS",
               "samples": [round(v, 1) for v in samples],
               "h2d_bytes_per_step": 8 * cells / args.steps,
               "d2h_bytes_per_step": 24 * cells / args.steps,
               "note": "lbm_init_density (8 B/cell H2D) + K x lbm_step + lbm_get_moments "
                       "(24 B/cell D2H), host arrays from lbm_host_alloc (page-locked), "
                       "wall clock; median of three timed passes"}
    lat.close()

    variants = {}
    # the other workloads' legs are single-GPU measurements: N = 1 only, so
    # that a scaling run times its replicas and nothing else
    if args.variants and rank == 0 and world == 1:
        for name, p in (("bf16dev", lbm.BF16DEV), ("fp16dev", lbm.FP16DEV)):
            v = lbm.Lattice(n, n, 0.85, precision=p, device=local, stream=stream.cuda_stream)
            v.init_density(rho0)
            v.step_async(args.warmup, lbm.IMPROVED, 0.8, 0.1)
            torch.cuda.synchronize()
            k = max(args.steps // 2, 1)
            s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s2.record(stream)
            v.step_async(k, lbm.IMPROVED, 0.8, 0.1)
            e2.record(stream)
            torch.cuda.synchronize()
            assert v.sync() == lbm.LBM_OK
            t_ms = s2.elapsed_time(e2)
            gbs = BYTES_PER_CELL[name] * cells / (t_ms * 1e-3 / k) / 1e9
            variants[name] = {"MLUPS": cells * k / (t_ms * 1e-3) / 1e6, "achieved_GBs": gbs,
                              "frac": gbs / peak, "bytes_per_cell": BYTES_PER_CELL[name]}
            v.close()

    # every forcing scheme of Table I and the MRT form, FP32, on a liquid slab
    # at the Maxwell densities of T = 0.9 Tc (Ladd's forcing diverges from
    # the 0.85 Tc spinodal start and from 0.85 Tc slabs); the headline is the
    # improved scheme
    schemes = {}
    if args.variants and rank == 0 and world == 1 and args.precision == "fp32":
        from paper_1204_4098_gb300 import inputs
        rg, rl, _ = lbm.maxwell(lbm.temperature(0.9))
        slab = inputs.slab_step(n, n, rg, rl)
        for name, sch, sigma in (("SC", lbm.SC, 0.0), ("EDM", lbm.EDM, 0.0),
                                 ("improved", lbm.IMPROVED, 0.1), ("noforce", lbm.NOFORCE, 0.0),
                                 ("EDM_Ce_1_over_tau", lbm.EDM_MOD, 0.0), ("Ladd", lbm.LADD, 0.0),
                                 ("MRT_improved", lbm.MRT, 0.1)):
            v = lbm.Lattice(n, n, 0.9, precision=lbm.FP32, device=local,
                            stream=stream.cuda_stream)
            if sch == lbm.MRT:
                v.set_mrt_rates(0.8, 1.1, 1.3)
            v.init_density(slab)
            v.step_async(args.warmup, sch, 0.8, sigma)
            torch.cuda.synchronize()
            k = max(args.steps // 2, 1)
            s2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s2.record(stream)
            v.step_async(k, sch, 0.8, sigma)
            e2.record(stream)
            torch.cuda.synchronize()
            st = v.sync()
            t_ms = s2.elapsed_time(e2)
            gbs = BYTES_PER_CELL["fp32"] * cells / (t_ms * 1e-3 / k) / 1e9
            schemes[name] = {"MLUPS": round(cells * k / (t_ms * 1e-3) / 1e6, 1),
                             "frac": round(gbs / peak, 4),
                             "status": lbm.STATUS_NAMES.get(st, st)}
            v.close()

    sweep_line = sweep512 = None
    if rank == 0 and world == 1 and not args.no_sweep:
        sweep_line = sweep_measure(128, 128, seed=4, device=local)
        sweep512 = sweep_batched_only(512, seed=4, device=local)

    warm_line = None
    if rank == 0 and world == 1 and not args.no_warmstart:
        warm_line = {"label": "reduced config 5: 6,000 training draws (nx = 32 slabs, cap 6e4 "
                              "steps; config 5: 11,000), 3 x 1500 epochs, the 256 held-out "
                              "256x256 points; cold sequential measured over all 256",
                     **warmstart_measure(6000, 1500, 256, device=local, train_max_steps=60000)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "bf16dev": "bf16", "fp16dev": "f16"}[
                    args.precision],
                "data": "synthetic", "config": workload_config(args),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches}
        if variants:
            line["storage_variants"] = variants
        if schemes:
            line["schemes_fp32"] = {"workload": f"{n}x{n} slab at the Maxwell densities, "
                                                "T = 0.9 Tc, tau = 0.8", **schemes}
        if sweep_line:
            line["batched_sweep"] = sweep_line
        if sweep512:
            line["batched_sweep_config4_512"] = sweep512
        if warm_line:
            line["warm_start"] = warm_line
        print(json.dumps(line), flush=True)


def _status_counts(res):
    names = {0: "active", 1: "converged", 2: "diverged", 3: "capped"}
    out = {}
    for r in res:
        out[names[r["status"]]] = out.get(names[r["status"]], 0) + 1
    return out


def _coex_agreement(a, b):
    """Max relative difference of rho_g and rho_l over runs converged in both."""
    both = [k for k in range(len(a)) if a[k]["status"] == 1 and b[k]["status"] == 1]
    if not both:
        return None, 0
    err = max(max(abs(a[k]["rho_g"] / b[k]["rho_g"] - 1), abs(a[k]["rho_l"] / b[k]["rho_l"] - 1))
              for k in both)
    return err, len(both)


def sweep_measure(n_inst, n_seq, seed=4, device=0):
    """Config-4 style sweep: n_inst instances (grid 32..512 x 128..512, T/Tc in
    [0.45, 0.95], tau in [0.6, 1.5], sigma in [0, 0.2], scheme in {SC, EDM,
    improved}) from the cold Maxwell step, batched to convergence, against
    sequential plain runs of the first n_seq of them."""
    import numpy as np

    from paper_1204_4098_gb300 import inputs, sweep
    inst = inputs.sweep_instances(n_inst, seed=seed)
    g, l = sweep.cold_start_profiles(inst)
    w = np.zeros(n_inst)
    res, stats, wall = sweep.run_batched(inst, g, l, w, device=device)
    seq, seq_wall = sweep.run_sequential(inst[:n_seq], g[:n_seq], l[:n_seq], w[:n_seq],
                                         device=device)
    agree, n_both = _coex_agreement(res[:n_seq], seq)
    # measured over every instance when n_seq == n_inst; otherwise scaled
    seq_total = seq_wall * n_inst / max(n_seq, 1)
    per = np.array([r["wall"] for r in seq])
    cells_steps = sum(d["nx"] * d["ny"] * r["steps"] for d, r in zip(inst, res))
    return {"instances": n_inst, "batched_wall_s": wall, "batched_gpu_s": stats["gpu_ms"] / 1e3,
            "instances_per_s": n_inst / wall,
            "batched_MLUPS": cells_steps / (stats["gpu_ms"] * 1e-3) / 1e6,
            "windows": stats["windows"], "status": _status_counts(res),
            "sequential_instances_timed": n_seq, "sequential_wall_s": seq_wall,
            "sequential_wall_s_all": seq_total,
            "sequential_measured_in_full": n_seq == n_inst,
            "sequential_per_instance_s": {"min": float(per.min()), "median": float(np.median(per)),
                                          "max": float(per.max())} if len(per) else None,
            "speedup_vs_sequential": seq_total / wall,
            "coexistence_max_rel_diff_vs_sequential": agree, "converged_in_both": n_both,
            "convergence_rule": "COEX: rho_g, rho_l (FP64 row means) change < max(1e-9, 8 ulp) "
                                "over two consecutive 1000-step windows; cap 2e5 steps",
            "init": "cold: Maxwell densities, sharp slab (rows [ny/4, 3ny/4) liquid)"}


def sweep_batched_only(n_inst, seed=4, device=0):
    """Config 4 at its full size (512 instances), batched only: the
    sequential baseline of this size is measured by --workload sweep (a
    sample, scaled), the 128-instance sweep of the default line measures it
    over every instance."""
    import numpy as np

    from paper_1204_4098_gb300 import inputs, sweep
    inst = inputs.sweep_instances(n_inst, seed=seed)
    g, l = sweep.cold_start_profiles(inst)
    res, stats, wall = sweep.run_batched(inst, g, l, np.zeros(n_inst), device=device)
    cells_steps = sum(d["nx"] * d["ny"] * r["steps"] for d, r in zip(inst, res))
    return {"instances": n_inst, "batched_wall_s": wall, "batched_gpu_s": stats["gpu_ms"] / 1e3,
            "instances_per_s": n_inst / wall,
            "batched_MLUPS": cells_steps / (stats["gpu_ms"] * 1e-3) / 1e6,
            "windows": stats["windows"], "status": _status_counts(res),
            "convergence_rule": "COEX (as the 128-instance sweep); cap 2e5 steps",
            "init": "cold: Maxwell densities, sharp slab (rows [ny/4, 3ny/4) liquid)"}


def run_sweep_workload(args, world, rank, local):
    """Config 4.  One GPU: batched vs sequential plain runs.  Under torchrun the
    instances are sharded across ranks (longest-processing-time on cells, no
    data-path collective), each rank runs its share as one batch, and the
    results are gathered on the host; value = all instances / slowest rank."""
    import numpy as np
    import torch

    from paper_1204_4098_gb300 import inputs, sweep
    torch.cuda.set_device(local)
    if world == 1:
        res = sweep_measure(args.sweep_instances, args.seq_sample, device=local)
        line = {"metric": METRIC, "workload": "batched parameter sweep (config 4)",
                "value": res["instances_per_s"], "unit": "instances/s", "n_gpus": world,
                "higher_is_better": True, "data": "synthetic", "dtype": "f32", **res}
        print(json.dumps(line), flush=True)
        return
    inst = inputs.sweep_instances(args.sweep_instances, seed=4)
    mine = sweep.shard(inst, world, rank)
    sub = [inst[i] for i in mine]
    g, l = sweep.cold_start_profiles(sub)
    dist_barrier(world)
    res, stats, wall = sweep.run_batched(sub, g, l, np.zeros(len(sub)), device=local)
    wall_max = dist_max(wall, world)
    everything = sweep.gather_results(mine, res, len(inst), world)
    if rank == 0:
        line = {"metric": METRIC, "workload": "batched parameter sweep (config 4), sharded",
                "value": len(inst) / wall_max, "unit": "instances/s", "n_gpus": world,
                "higher_is_better": True, "scaling": "strong", "data": "synthetic",
                "dtype": "f32", "instances": len(inst), "wall_s_max_over_ranks": wall_max,
                "status": _status_counts(everything)}
        print(json.dumps(line), flush=True)


def warmstart_measure(train_draws, epochs, held_out, device=0, seq_all=True, seed_train=40,
                      seed_held=41, train_max_steps=100000, trend_tol=None):
    """Config 5: train the network on converged cold runs of narrow slabs,
    then start held-out points on 256 x 256 grids from its predictions and
    compare the whole sweep with cold batched runs and with cold sequential
    plain runs, all stopped by the same TREND rule."""
    import numpy as np

    from paper_1204_4098_gb300 import inputs, lbm, sweep, warmstart
    t0 = time.perf_counter()
    X, Y, info = warmstart.training_data(train_draws, seed=seed_train, max_steps=train_max_steps,
                                         trend_tol=trend_tol)
    data_s = time.perf_counter() - t0
    model = warmstart.train(X, Y, stages=((epochs, 2e-3), (epochs, 5e-4), (epochs, 1e-4)),
                            batch=128, seed=1, device=device)
    held = inputs.sweep_instances(held_out, seed=seed_held, nx_range=(256, 256),
                                  ny_range=(256, 256))
    warm, winfo = warmstart.run_warm(held, model, device=device, trend_tol=trend_tol)
    cold, cinfo = warmstart.run_cold_batched(held, device=device, trend_tol=trend_tol)
    g, l = sweep.cold_start_profiles(held)
    ns = len(held) if seq_all else min(32, len(held))
    seq, seq_wall = sweep.run_sequential(held[:ns], g[:ns], l[:ns], np.zeros(ns), device=device,
                                         conv=lbm.CONV_TREND, trend_tol=trend_tol)
    seq_all_s = seq_wall * len(held) / ns
    err, n_both = _coex_agreement(warm, cold)
    err_seq, n_both_seq = _coex_agreement(warm[:ns], seq)
    both = [k for k in range(len(held)) if warm[k]["status"] == 1 and cold[k]["status"] == 1]
    mean = lambda rs: float(np.mean([rs[k]["steps"] for k in both])) if both else None
    t_warm, s_warm = warmstart.time_to_answer(warm, winfo, cold, among=both)
    warm_gpu, cold_gpu = winfo["gpu_ms"] / 1e3, cinfo["gpu_ms"] / 1e3
    arbiter = _long_run_arbiter(held, warm, cold, both, device)
    return {"held_out": len(held), "grid": "256x256",
            "trend_tol": sweep.TREND_TOL if trend_tol is None else trend_tol,
            "rule": "TREND: rho_g, rho_l settled to 1e-4 over the last nine windows (range of "
                    "the last six, geometric extrapolation of three-window block means), warm, "
                    "cold batched and cold sequential alike; fallback: limits extrapolated from "
                    "the first three windows > 1e-2 from the prediction, or divergence",
            "training": {**info, "data_wall_s": data_s, "train_loss": model.train_loss,
                         "train_s": model.train_seconds, "epochs": [epochs] * 3,
                         "learning_rates": [2e-3, 5e-4, 1e-4]},
            "warm_batched": {"gpu_s": warm_gpu, "wall_s": winfo["wall"],
                             "fallbacks": winfo["fallbacks"], "status": _status_counts(warm),
                             "mean_steps_converged_both": mean(warm)},
            "cold_batched": {"gpu_s": cold_gpu, "wall_s": cinfo["wall"],
                             "status": _status_counts(cold), "mean_steps_converged_both": mean(cold)},
            "cold_sequential": {"instances_timed": ns, "wall_s": seq_wall,
                                "wall_s_all": seq_all_s, "measured_in_full": ns == len(held),
                                "status": _status_counts(seq)},
            "whole_sweep_cold_batched_over_warm_batched": cold_gpu / warm_gpu,
            "whole_sweep_cold_sequential_over_warm_batched": seq_all_s / warm_gpu,
            "coexistence_max_rel_err_warm_vs_cold_batched": err,
            "converged_in_both": n_both,
            "coexistence_max_rel_err_warm_vs_cold_sequential": err_seq,
            "converged_in_both_sequential": n_both_seq,
            "retrospective_time_to_answer_warm_gpu_s": t_warm,
            "retrospective_mean_steps_to_answer_warm": s_warm,
            "long_run_arbiter": arbiter}


def _long_run_arbiter(held, warm, cold, both, device, limit=5e-4, steps=150000):
    """Runs converged in both whose warm and cold answers differ by more than
    `limit` are run again from the cold start for `steps` steps (no stop):
    how far each answer is from that long run says which of the two stopped
    early (outside the timed sweeps)."""
    import numpy as np

    from paper_1204_4098_gb300 import lbm, sweep
    rel = lambda a, b: max(abs(a["rho_g"] / b["rho_g"] - 1), abs(a["rho_l"] / b["rho_l"] - 1))
    ks = [k for k in both if rel(warm[k], cold[k]) > limit]
    if not ks:
        return {"runs": 0, "limit": limit}
    sub = [held[k] for k in ks]
    g, l = sweep.cold_start_profiles(sub)
    with lbm.Batch(sub, window=1000, tol=0.0, max_steps=steps, conv=lbm.CONV_NONE,
                   device=device) as b:
        b.init_slabs(g, l, np.zeros(len(sub)))
        b.run()
        long = b.results()
    return {"runs": len(ks), "limit": limit, "steps": steps,
            "warm_vs_long_max": max(rel(warm[k], r) for k, r in zip(ks, long)),
            "cold_vs_long_max": max(rel(cold[k], r) for k, r in zip(ks, long)),
            "warm_vs_cold_max": max(rel(warm[k], cold[k]) for k in ks)}


def run_warmstart_workload(args, world, rank, local):
    """Config 5 in full (about 11,000 training draws, 256 held-out points)."""
    import torch
    torch.cuda.set_device(local)
    res = warmstart_measure(args.train_draws, args.epochs, args.held_out, device=local,
                            trend_tol=args.trend_tol)
    line = {"metric": METRIC, "workload": "learned warm start (config 5)",
            "value": res["whole_sweep_cold_sequential_over_warm_batched"],
            "unit": "x less whole-sweep time: warm batched GPU vs cold sequential plain runs",
            "higher_is_better": True, "n_gpus": world, "data": "synthetic", "dtype": "f32",
            **res}
    print(json.dumps(line), flush=True)


def run_band_workload(args, world, rank, local):
    """Strong scaling of one lattice: the n x n workload split into `world`
    y-slabs (halo.band_partition), one per rank, each step followed by the
    halo exchange (two rows x 9 populations to each neighbour, NCCL point to
    point on device buffers).  At N = 1 the band exchanges with itself (the
    periodic wrap).  For N > 1 the exchange runs on a second stream while the
    interior rows are computed; the other path is timed beside it.
    value = all cells x steps / the slowest rank's time."""
    import torch
    import torch.distributed as dist

    from paper_1204_4098_gb300 import halo, lbm
    torch.cuda.set_device(local)
    group = None
    if world > 1:
        group = dist.new_group(backend="nccl")
    n = args.n
    rho0, _ = workload_density(n, 0)
    band = halo.BandLattice(n, n, 0.85, rho0, rank=rank, world=world, device=local,
                            group=group)
    def timed(overlap):
        band.step(args.warmup, lbm.IMPROVED, 0.8, 0.1, overlap=overlap)
        torch.cuda.synchronize()
        dist_barrier(world)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches0 = lbm.launch_count()
        start.record(band.stream)
        st = band.step(args.steps, lbm.IMPROVED, 0.8, 0.1, overlap=overlap)
        end.record(band.stream)
        torch.cuda.synchronize()
        dist_barrier(world)
        assert st == lbm.LBM_OK
        return dist_max(start.elapsed_time(end), world), lbm.launch_count() - launches0

    ms_other, _ = timed(world == 1)
    ms, launches = timed(world > 1)  # the default of halo.BandLattice.step
    if rank == 0:
        line = {"metric": METRIC, "workload": f"{n}x{n} single lattice in {world} y-slabs "
                                              "with halo exchange (strong scaling)",
                "value": n * n * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
                "data": "synthetic", "dtype": "f32", "rows_per_rank": band.rows,
                "halo_bytes_per_message": band.lat.halo_bytes(),
                "exchange": "overlapped with the interior rows (boundary rows first)"
                            if world > 1 else "self-exchange after the step (nothing to hide)",
                ("without_overlap_MLUPS" if world > 1 else "with_overlap_MLUPS"):
                    n * n * args.steps / (ms_other * 1e-3) / 1e6,
                "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    band.close()


def run_droplets_workload(args, world, rank, local):
    """Config 2: droplets on 256 x 256 (R0 = 20, 30, 40, 50; W = 5) for every
    T/Tc in {0.6, 0.7, 0.8, 0.9}, tau in {0.6, 1.0, 1.5} and scheme (Shan-Chen,
    EDM, improved with sigma = 0, 0.05, 0.1, 0.15, 0.105), 2e4 steps each, in
    one batch; Laplace fits and coexistence per sweep point."""
    import torch

    from paper_1204_4098_gb300 import droplets, lbm
    torch.cuda.set_device(local)
    inst = droplets.laplace_instances()
    res, info = droplets.run(inst, args.droplet_steps)
    fits = droplets.laplace_fits(inst, res)
    names = {lbm.SC: "SC", lbm.EDM: "EDM", lbm.IMPROVED: "improved"}
    table = []
    for (t, tau, sch, sg), f in sorted(fits.items()):
        runs = [r for d, r in zip(inst, res)
                if (d["T_over_Tc"], d["tau"], d["scheme"], d["sigma"]) == (t, tau, sch, sg)]
        row = {"T_over_Tc": t, "tau": tau, "scheme": names[sch], "sigma": sg,
               "stable": f is not None,
               "diverged": sum(droplets.unstable(r) for r in runs),
               "dissolved": sum((not droplets.unstable(r)) and droplets.vanished(r)
                                for r in runs)}
        if f is not None:
            row.update({k: f[k] for k in ("surface_tension", "intercept", "intercept_se",
                                          "r2", "max_speed")})
            row["rho_l_R50"], row["rho_g_R50"] = f["rho_in"][-1], f["rho_out"][-1]
        table.append(row)
    cells_steps = sum(d["nx"] * d["ny"] * r["steps"] for d, r in zip(inst, res))
    stable = [r for r in table if r["stable"]]
    line = {"metric": METRIC, "workload": "droplets and Laplace's law (config 2)",
            "value": cells_steps / (info["gpu_ms"] * 1e-3) / 1e6, "unit": "MLUPS (batched)",
            "higher_is_better": True, "n_gpus": world, "data": "synthetic", "dtype": "f32",
            "runs": len(inst), "steps": args.droplet_steps, "gpu_s": info["gpu_ms"] / 1e3,
            "wall_s": info["wall"], "status": _status_counts(res),
            "laplace_points": len(table), "laplace_stable": len(stable),
            "laplace_min_r2": min((r["r2"] for r in stable), default=None),
            "laplace_median_r2": float(sorted(r["r2"] for r in stable)[len(stable) // 2])
            if stable else None,
            "table": table}
    print(json.dumps(line), flush=True)


def run_stability_workload(args, world, rank, local):
    """Figs. 1, 2, 7: lowest stable T/Tc of a 200 x 200 droplet (r0 = 30, initial
    interface width W = 4 by default, Maxwell densities, Tc = 0.094 as
    printed, started at rest: zero actual velocity) per scheme and tau, on a
    T/Tc ladder 0.95 .. 0.45 in steps of 0.01, in one batch."""
    import json as _json

    import numpy as np
    import torch

    from paper_1204_4098_gb300 import droplets, lbm
    torch.cuda.set_device(local)
    schemes = ((lbm.SC, 0.0), (lbm.EDM, 0.0), (lbm.EDM_MOD, 0.0), (lbm.IMPROVED, 0.0),
               (lbm.IMPROVED, 0.105))
    taus = (0.6, 0.7, 0.8, 0.9)
    temps = np.round(np.arange(0.95, 0.4499, -0.01), 2)
    inst = droplets.stability_instances(schemes, taus, temps)
    res, info = droplets.run(inst, args.stability_steps, W=args.stability_width, tc_mode=1,
                             at_rest=True)
    th = droplets.thresholds(inst, res)
    names = {lbm.SC: "SC", lbm.EDM: "EDM", lbm.EDM_MOD: "EDM_Ce=1/tau",
             lbm.IMPROVED: "improved"}
    with open(os.path.join(ROOT, "tests", "golden", "paper_values.json")) as f:
        paper = _json.load(f)
    cells_steps = sum(d["nx"] * d["ny"] * r["steps"] for d, r in zip(inst, res))
    line = {"metric": METRIC, "workload": "droplet stability thresholds (Figs. 1, 2, 7)",
            "value": cells_steps / (info["gpu_ms"] * 1e-3) / 1e6, "unit": "MLUPS (batched)",
            "higher_is_better": True, "n_gpus": world, "data": "synthetic", "dtype": "f32",
            "runs": len(inst), "steps": args.stability_steps, "gpu_s": info["gpu_ms"] / 1e3,
            "wall_s": info["wall"], "status": _status_counts(res),
            "criterion": f"diverged, or max |v| > {droplets.UNSTABLE_SPEED} after the budget",
            "initial_width": args.stability_width,
            "initial_velocity": "at rest: u = -F/(2 rho), zero actual velocity (Table I)",
            "lowest_stable_T_over_Tc": [
                {"scheme": names[s], "sigma": sg, "tau": tau, "T_min": t}
                for (s, sg, tau), t in sorted(th.items())],
            "paper": {"tau0.6": paper["stability_threshold_tau06"]["value"],
                      "tau0.7": paper["stability_threshold_modified_edm"]["value"]}}
    print(json.dumps(line), flush=True)


def run_calibrate_workload(args, world, rank, local):
    """Sec. IV B automated: sigma*(T) where converged flat-interface slabs of
    the improved scheme meet the Maxwell vapour density, T/Tc 0.65 .. 0.9."""
    import numpy as np
    import torch

    from paper_1204_4098_gb300 import calibrate
    torch.cuda.set_device(local)
    temps = np.round(np.arange(0.65, 0.9001, 0.05), 2)
    t0 = time.perf_counter()
    out, info = calibrate.sigma_star(temps)
    stars = [r["sigma_star"] for r in out if r["sigma_star"] is not None]
    line = {"metric": METRIC, "workload": "sigma calibration against Maxwell (Sec. IV B)",
            "value": float(np.mean(stars)) if stars else None,
            "unit": "mean sigma* over T (paper: 0.105)", "higher_is_better": None,
            "n_gpus": world, "data": "synthetic", "dtype": "f32", "gpu_s": info["gpu_s"],
            "wall_s": time.perf_counter() - t0,
            "sigma_star": [{"T_over_Tc": r["T_over_Tc"], "sigma_star": r["sigma_star"],
                            "eps_star": r["eps_star"]} for r in out],
            "curves": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--precision", choices=tuple(BYTES_PER_CELL), default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", action="store_true", default=True)
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--ref-side", type=int, default=1024)
    ap.add_argument("--workload", choices=("roofline", "sweep", "warmstart", "droplets",
                                           "stability", "calibrate", "band"),
                    default="roofline")
    ap.add_argument("--droplet-steps", type=int, default=20000)
    ap.add_argument("--stability-steps", type=int, default=20000)
    ap.add_argument("--stability-width", type=float, default=4.0)
    ap.add_argument("--sweep-instances", type=int, default=512)
    ap.add_argument("--seq-sample", type=int, default=32)
    ap.add_argument("--train-draws", type=int, default=11000)
    ap.add_argument("--epochs", type=int, default=1500)
    ap.add_argument("--held-out", type=int, default=256)
    ap.add_argument("--trend-tol", type=float, default=None,
                    help="TREND stopping bound of the warm-start workload (default 1e-4)")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-warmstart", action="store_true")
    ap.add_argument("--kernel-variant", choices=("auto", "register", "pair", "staged"),
                    default="auto", help="step kernel of the roofline run")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "sweep":
        run_sweep_workload(args, world, rank, local)
    elif args.workload == "warmstart":
        run_warmstart_workload(args, world, rank, local)
    elif args.workload == "droplets":
        run_droplets_workload(args, world, rank, local)
    elif args.workload == "stability":
        run_stability_workload(args, world, rank, local)
    elif args.workload == "calibrate":
        run_calibrate_workload(args, world, rank, local)
    elif args.workload == "band":
        run_band_workload(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
