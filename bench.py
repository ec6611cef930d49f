"""Benchmark: batched Shen solves (Helmholtz + biharmonic per Fourier mode) on GB300.

One step = one Helmholtz solve and one biharmonic solve of every mode of the
workload (two right-hand-side fields in, two solution fields out), through the C
ABI of libshensolve.  Default workload: N = 1024 Chebyshev modes, 1024 x 1024
Fourier grid (513 x 1024 = 525,312 modes), nu = 1/2000, dt = 1e-4.

Metric: Shen solves*N/s = (systems solved per step * N) / step time.
Prints one JSON line (rank 0).  `--impl reference` times the oracle's O(N) C code
(the paper's algorithms, OpenMP) on the host cores instead.
"""
import argparse
import ctypes
import datetime
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "small": dict(N=64, Nx=32, Nz=32, nu=1 / 180, dt=1e-3),
    "retau180": dict(N=128, Nx=128, Nz=128, nu=1 / 180, dt=5e-4),
    "n1024": dict(N=1024, Nx=1024, Nz=1024, nu=1 / 2000, dt=1e-4),
    "large": dict(N=1536, Nx=2048, Nz=1536, nu=1 / 2000, dt=5e-5),
    # profiling cases: N = 1024 columns on a 128 x 128 grid (136 MB per field, > L2; under
    # one wave of blocks) and on a 256 x 256 grid (540 MB per field, several waves)
    "n1024s": dict(N=1024, Nx=128, Nz=128, nu=1 / 2000, dt=1e-4),
    "n1024q": dict(N=1024, Nx=256, Nz=256, nu=1 / 2000, dt=1e-4),
    # 4096 channels with uneven N (64..512), grids 16..64, nu in [1e-4, 1e-2], dt in [1e-4, 1e-2]
    "batch": dict(n_inst=4096, seed=5),
}
METRIC = "Shen solves*N/s (Helmholtz + biharmonic, all modes)"
LEAN_WORKLOADS = {"large"}
BYTES_PER_ROW = 32          # algorithmic bytes per complex row of one solve: read f + write u


# arithmetic of each solve path (all read and write complex128 fields)
DTYPES = {"fp64": "f64", "df": "f32x2 (float-float)", "df_r1": "f32 sweeps + f32x2 refinement",
          "df_r2": "f32 sweeps + f32x2 refinement", "fp32_r1": "f32 sweeps + f64 refinement",
          "fp32_r2": "f32 sweeps + f64 refinement", "fp64_r1": "f64 sweeps + f64x2 refinement"}


def dtype_of(prec):
    names = {DTYPES.get(p, p) for p in prec.values()}
    if len(names) == 1:
        return names.pop()
    return ", ".join(f"{k}: {DTYPES.get(v, v)}" for k, v in sorted(prec.items()))


def n_modes_of(w):
    return (w["Nx"] // 2 + 1) * w["Nz"]


# CUDA sources each profiled kernel is built from (its traffic figure is valid while they hash
# to the value stored with it)
TRAFFIC_SOURCES = {
    "df": ("kernels_df.cu", "chains.cuh", "df.cuh"),
    "velocity": ("velocity.cu", "chains.cuh", "df.cuh"),
    "matvec": ("matvec_df.cu", "df.cuh"),
    "transform": ("transform.cu", "colgroup.cuh", "df.cuh"),
}


TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def traffic_group(kind):
    head = kind.split(":")[0]
    if head.startswith("velocity"):
        return "velocity"
    if head.startswith("matvec"):
        return "matvec"
    if head == "transform":
        return "transform"
    return "df"


def sources_sha1(names):
    """Hash of the kernels' code: the named CUDA sources with their comments removed (so
    that a change of wording does not retire a capture of unchanged code)."""
    import hashlib
    import re
    h = hashlib.sha1()
    for name in sorted(names):
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_1701_03787_gb300", "csrc", name)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(text.encode())
    return h.hexdigest()


def measured_traffic(kind, rows):
    """DRAM bytes of one launch of `kind` ("problem:precision") over `rows` complex rows,
    scaled from the per-row figure of an ncu capture (profiles/traffic.json); None if the
    kernel's CUDA sources have changed since that capture."""
    path = TRAFFIC_PATH
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        t = json.load(fh)
    entry = t.get("bytes_per_row", {}).get(kind)
    group = traffic_group(kind)
    hashes = t.get("sources_sha1")
    if entry is None or not isinstance(hashes, dict) or hashes.get(group) != sources_sha1(TRAFFIC_SOURCES[group]):
        return None
    return entry * rows


# kernel name (as ncu prints it) -> traffic kinds its per-launch bytes stand for
TRAFFIC_KERNELS = (
    (r"bih_df_kernel<0>", ("biharmonic:df",)),
    (r"helm_df_kernel<0>", ("helmholtz:df",)),
    (r"velocity_df_kernel", ("velocity:df",)),
    (r"matvec_helmholtz_df_kernel<0>", ("matvec_helmholtz:df",)),
    (r"matvec_biharmonic_df_kernel<0>", ("matvec_biharmonic:df",)),
    (r"transform_kernel<0, 0, (0|false)>", ("transform:inverse_chebyshev",)),
    (r"transform_kernel<0, 1, (0|false)>", ("transform:inverse_dirichlet",)),
    (r"transform_kernel<0, 2, (0|false)>", ("transform:inverse_biharmonic",)),
    (r"transform_kernel<1, 0, (0|false)>", ("transform:scalar_chebyshev",)),
    (r"transform_kernel<1, 1, (0|false)>", ("transform:scalar_dirichlet",)),
    (r"transform_kernel<1, 2, (0|false)>", ("transform:scalar_biharmonic",)),
    (r"transform_kernel<2, 0, (0|false)>", ("transform:forward_chebyshev",)),
    (r"transform_kernel<2, 1, (0|false)>", ("transform:forward_dirichlet",)),
    (r"transform_kernel<2, 2, (0|false)>", ("transform:forward_biharmonic",)),
)


def write_traffic(csv_paths, w):
    """Rewrite profiles/traffic.json from ncu CSV launch lists with dram__bytes_read.sum and
    dram__bytes_write.sum of the kernels above (one CSV per capture, e.g. one per kernel),
    taken on workload `w`: bytes per complex row (averaged over the captured launches of each
    kernel), stamped with the current hashes of each group's sources."""
    import csv
    import re
    if isinstance(csv_paths, str):
        csv_paths = [csv_paths]
    per_launch = {}
    for f_i, csv_path in enumerate(csv_paths):
        with open(csv_path) as fh:
            lines = [ln for ln in fh if ln.startswith('"')]
        rows = list(csv.reader(lines))
        if not rows:
            continue
        hdr = rows[0]
        c_id, c_name = hdr.index("ID"), hdr.index("Kernel Name")
        c_metric, c_val = hdr.index("Metric Name"), hdr.index("Metric Value")
        for r in rows[1:]:
            if r[c_metric] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                key = (f_i, r[c_id])                      # launch IDs restart in every capture
                name, b = per_launch.get(key, (r[c_name], 0.0))
                per_launch[key] = (name, b + float(r[c_val].replace(",", "")))
    n_rows = n_modes_of(w) * w["N"]
    counts, per_kind = {}, {}
    for pat, kinds in TRAFFIC_KERNELS:
        launches = [b for name, b in per_launch.values() if re.search(pat, name)]
        if launches:
            counts[pat] = len(launches)
            for k in kinds:
                per_kind[k] = per_kind.get(k, 0.0) + sum(launches) / len(launches)
    bpr = {k: round(v / n_rows, 2) for k, v in sorted(per_kind.items())}
    out = {"note": "DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per complex row (n_modes * N rows) "
                   "for one launch, from an ncu capture "
                   f"on the N={w['N']}, {w['Nx']}x{w['Nz']} workload, written by bench.py --write-traffic; each "
                   "figure is valid while its kernels' CUDA sources (comments removed) hash to sources_sha1[group] "
                   "(groups and files: bench.py TRAFFIC_SOURCES)",
           "workload": {k: w[k] for k in ("N", "Nx", "Nz")},
           "launches": {pat: counts[pat] for pat, _ in TRAFFIC_KERNELS if counts.get(pat)},
           "sources_sha1": {g: sources_sha1(names) for g, names in TRAFFIC_SOURCES.items()},
           "bytes_per_row": bpr}
    with open(TRAFFIC_PATH, "w") as fh:
        json.dump(out, fh, indent=2)
        fh.write("\n")
    return out


def gpu_pci_id(dev):
    """PCI bus id of CUDA device `dev` in NVML's format, or None."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    if not all(hasattr(p, a) for a in ("pci_domain_id", "pci_bus_id", "pci_device_id")):
        return None
    return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"


def _mask_bits(mask):
    bits = 8 * ctypes.sizeof(ctypes.c_ulong)
    return {w * bits + b for w in range(len(mask)) for b in range(bits) if (mask[w] >> b) & 1}


def bind_gpu_local_host(pci):
    """Place this process next to the GPU: run it on the CPUs NVML reports as local to the
    GPU, and prefer the GPU's NUMA node for its host memory (so that pinned buffers land
    there).  NVML is only queried; the binding affects this process alone.  Returns a
    description of the host topology seen."""
    info = {"cpus_allowed": len(os.sched_getaffinity(0))}
    try:
        with open("/proc/self/status") as fh:
            for line in fh:
                if line.startswith("Mems_allowed_list"):
                    info["mems_allowed"] = line.split(":", 1)[1].strip()
        info["numa_nodes"] = sorted(int(d[4:]) for d in os.listdir("/sys/devices/system/node")
                                    if d.startswith("node") and d[4:].isdigit())
    except Exception:
        pass
    try:
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            return info
        try:
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), ctypes.byref(h)) != 0:
                return info
            cmask = (ctypes.c_ulong * 64)()
            cpus = _mask_bits(cmask) if nv.nvmlDeviceGetCpuAffinity(h, 64, cmask) == 0 else set()
            nmask = (ctypes.c_ulong * 4)()
            nodes = _mask_bits(nmask) if nv.nvmlDeviceGetMemoryAffinity(h, 4, nmask, 0) == 0 else set()
        finally:
            nv.nvmlShutdown()
        cpus &= os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus)
            info["cpus_gpu_local"] = len(cpus)
        if nodes:
            info["gpu_numa_nodes"] = sorted(nodes)
            # set_mempolicy(MPOL_PREFERRED, node): later first touches prefer the GPU's node
            libc = ctypes.CDLL(None, use_errno=True)
            node = min(nodes)
            m = (ctypes.c_ulong * 16)()
            m[node // 64] = 1 << (node % 64)
            import platform
            nr = {"aarch64": 237, "x86_64": 238}.get(platform.machine())    # set_mempolicy
            if nr is not None:
                ok = libc.syscall(nr, 1, m, ctypes.c_ulong(16 * 64 + 1)) == 0
                info["mempolicy_preferred_node"] = node if ok else None
    except Exception as ex:
        info["error"] = type(ex).__name__
    return info


def max_over_ranks(values, pg, device):
    """Element-wise maximum of a list of floats over all ranks (the list itself at one rank)."""
    if pg is None:
        return list(values)
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons every 100 ms; only the samples whose
    timestamps fall inside the timed region (mark_begin .. mark_end) are kept."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu = gpu_id
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark_begin(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                    if self.t0 and self.t1 and not (self.t0 <= ts <= self.t1):
                        continue
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, precision_note, seconds_target=8.0, seed=0):
    """The oracle's O(N) C solvers (paper's algorithms, OpenMP over modes) on a bounded
    sample of the workload's modes; returns solves*N/s."""
    from oracle import on
    from oracle import solve as so
    from paper_1701_03787_gb300 import inputs
    N = w["N"]
    c = so.c_of(w["nu"], w["dt"])
    z2_all = so.mode_z2(w["Nx"], w["Nz"])
    n_sample = min(z2_all.size, max(1024, int(2 ** 26 // (16 * N))))       # ~64 MB per field
    idx = np.linspace(0, z2_all.size - 1, n_sample).astype(np.int64)
    z2 = z2_all[idx]
    F = inputs.rhs_numpy(n_sample, N, seed)
    on.solve_modes("helmholtz", N, z2, c, F[:8])                             # load / warm
    reps, t_total, t0 = 0, 0.0, time.perf_counter()
    while True:
        t = time.perf_counter()
        on.solve_modes("helmholtz", N, z2, c, F)
        on.solve_modes("biharmonic", N, z2, c, F)
        t_total += time.perf_counter() - t
        reps += 1
        if time.perf_counter() - t0 > seconds_target or reps >= 50:
            break
    value = reps * 2 * n_sample * N / t_total
    cores = on.max_threads()
    # the same solves on one core (a quarter of the sample, once)
    n1 = max(64, n_sample // 4)
    prev = on.set_threads(1)
    try:
        t = time.perf_counter()
        on.solve_modes("helmholtz", N, z2[:n1], c, F[:n1])
        on.solve_modes("biharmonic", N, z2[:n1], c, F[:n1])
        single = 2 * n1 * N / (time.perf_counter() - t)
    finally:
        on.set_threads(prev)
    return {"value": value, "unit": "solves*N/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_sample} of {z2_all.size} modes (evenly spaced), Helmholtz + biharmonic, "
                      f"{reps} repetitions, O(N) C oracle (Sec. 4 algorithms), float64",
            "single_core": {"value": single, "unit": "solves*N/s", "cores": 1,
                            "sample": f"the first {n1} modes of that sample, once"}}


def cpu_transforms(N, n_cols=256, seed=0):
    """The transforms oracle (oracle/transforms.py: dense basis matrices at the Gauss points,
    numpy / BLAS on the host cores) on `n_cols` columns of N: complex points per second of the
    inverse transform and of the scalar products in the Dirichlet space."""
    from oracle import transforms as tr
    from paper_1701_03787_gb300 import inputs
    C = inputs.rhs_numpy(n_cols, N, seed)
    C[:, N - 2:] = 0
    tr.inverse("dirichlet", C[:2])                                      # warm (basis matrices)
    tr.scalar("dirichlet", C[:2])
    out = {}
    for kind, fn in (("inverse_dirichlet", tr.inverse), ("scalar_dirichlet", tr.scalar)):
        t = time.perf_counter()
        fn("dirichlet", C)
        out[kind] = {"points_per_s": n_cols * N / (time.perf_counter() - t)}
    out["sample"] = f"{n_cols} columns of N = {N}, dense float64 matrices (O(N^2) per column), numpy BLAS"
    out["cores"] = len(os.sched_getaffinity(0))
    return out


def cpu_baseline_batch(w, seconds_target=8.0, seed=0):
    """The oracle's O(N) C solvers on a bounded sample of the batching workload: every
    mode of evenly spaced instances, until about `seconds_target` of solving."""
    from oracle import on
    from oracle import solve as so
    from paper_1701_03787_gb300 import inputs
    insts = inputs.batch_instances(w["n_inst"], seed=w["seed"])
    picks = insts[::max(1, len(insts) // 256)]
    rows, t_total, n_done = 0, 0.0, 0
    t0 = time.perf_counter()
    for inst in picks:
        z2 = so.mode_z2(inst["Nx"], inst["Nz"], inst.get("Lx", 2 * math.pi), inst.get("Lz", math.pi))
        F = inputs.rhs_numpy(z2.size, inst["N"], seed + n_done)
        c = so.c_of(inst["nu"], inst["dt"])
        t = time.perf_counter()
        on.solve_modes("helmholtz", inst["N"], z2, c, F)
        on.solve_modes("biharmonic", inst["N"], z2, c, F)
        t_total += time.perf_counter() - t
        rows += 2 * z2.size * inst["N"]
        n_done += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    return {"value": rows / t_total, "unit": "solves*N/s", "cores": on.max_threads(), "kind": "oracle",
            "sample": f"all modes of {n_done} of {len(insts)} instances (evenly spaced), Helmholtz + biharmonic, "
                      f"O(N) C oracle (Sec. 4 algorithms), float64"}


def oracle_errors(w, F_h, F_b, results, modes, refined_modes):
    """Error of GPU results against the oracle on sampled modes.  results: {path: (U_h, U_b)},
    rows aligned with `modes` (global mode indices).  Every path against the O(N) C oracle
    (the paper's algorithm in float64) on all of `modes`, and against the refined reference
    (the O(N) solve refined with a longdouble residual of the exactly evaluated matrices) on
    `refined_modes`: max, median and field-level relative L2."""
    from oracle import on
    from oracle import solve as so
    from oracle import structured as st
    N = w["N"]
    c = so.c_of(w["nu"], w["dt"])
    z2 = so.mode_z2(w["Nx"], w["Nz"])
    pos = {m: i for i, m in enumerate(modes)}
    ref_rows = [pos[m] for m in refined_modes]
    out = {"n_modes_checked": len(modes), "n_refined": len(ref_rows)}
    for problem, F in (("helmholtz", F_h), ("biharmonic", F_b)):
        n = so.n_unknowns(problem, N)
        R = on.solve_modes(problem, N, z2[modes], c, F)
        Rr = st.solve_ref(problem, N, z2[refined_modes], c, F[ref_rows])
        for path, (U_h, U_b) in results.items():
            U = U_h if problem == "helmholtz" else U_b
            errs = [so.rel_l2(U[i, :n], R[i, :n]) for i in range(len(modes))]
            ref_errs = [so.rel_l2(U[i, :n], Rr[j, :n]) for j, i in enumerate(ref_rows)]
            num = sum(float(np.sum(np.abs(U[i, :n] - Rr[j, :n]) ** 2)) for j, i in enumerate(ref_rows))
            den = sum(float(np.sum(np.abs(Rr[j, :n]) ** 2)) for j in range(len(ref_rows)))
            out.setdefault(path, {})[problem] = {
                "vs_on_max": float(max(errs)), "vs_on_median": float(np.median(errs)),
                "vs_refined_max": float(max(ref_errs)), "vs_refined_median": float(np.median(ref_errs)),
                "vs_refined_field": math.sqrt(num / den)}
    return out


# Fastest path per problem that meets the 1e-10 bar (see the GPU parity tests).
AUTO_PRECISION = {"helmholtz": "df", "biharmonic": "df"}


def resolve_precision(spec):
    """Per-problem precisions of the step.  The fused refinement kernels (fp32_r1, df_r1)
    serve the Helmholtz problem only; the biharmonic solve then runs in float-float, the
    fastest biharmonic path that meets the 1e-10 bar."""
    if spec == "auto":
        return dict(AUTO_PRECISION)
    if spec in ("fp32_r1", "df_r1"):
        return {"helmholtz": spec, "biharmonic": "df"}
    return {"helmholtz": spec, "biharmonic": spec}


def run_reference(args, w):
    """The oracle's O(N) C code (the paper's algorithms, OpenMP over modes) as the reference
    arm.  Every step solves a bounded sample of the workload (both problems), so that the
    whole --steps K --warmup W run takes seconds to a minute; W steps run untimed, then K
    steps are timed one by one with a wall clock.  value and ms_per_step are those of the
    sampled steps; the time a whole-workload step would take at that rate is reported
    separately and labelled as extrapolated."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import on
    from oracle import solve as so
    from paper_1701_03787_gb300 import inputs
    cases = []                                      # (N, z2, c, F) per solve batch of a step
    if "n_inst" in w:
        insts = inputs.batch_instances(w["n_inst"], seed=w["seed"])
        full_rows = sum((d["Nx"] // 2 + 1) * d["Nz"] * d["N"] for d in insts)
        picks = insts[:: max(1, len(insts) // 64)]
        for i, d in enumerate(picks):
            z2 = so.mode_z2(d["Nx"], d["Nz"])
            cases.append((d["N"], z2, so.c_of(d["nu"], d["dt"]), inputs.rhs_numpy(z2.size, d["N"], i)))
        desc = f"all modes of {len(picks)} of {len(insts)} instances (every {max(1, len(insts) // 64)}th)"
    else:
        N = w["N"]
        z2_all = so.mode_z2(w["Nx"], w["Nz"])
        full_rows = z2_all.size * N
        n_sample = min(z2_all.size, max(1024, int(2 ** 25 // N)))       # 32 Mi rows: ~0.2 s per step
        idx = np.linspace(0, z2_all.size - 1, n_sample).astype(np.int64)
        cases.append((N, z2_all[idx], so.c_of(w["nu"], w["dt"]), inputs.rhs_numpy(n_sample, N, 0)))
        desc = f"{n_sample} of {z2_all.size} modes (evenly spaced)"
    rows = sum(z2.size * N_ for N_, z2, _, _ in cases)

    def one_step():
        for N_, z2, c, F in cases:
            on.solve_modes("helmholtz", N_, z2, c, F)
            on.solve_modes("biharmonic", N_, z2, c, F)

    for _ in range(max(args.warmup, 1)):
        one_step()
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        one_step()
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = args.steps * 2 * rows / total
    cores = on.max_threads()
    base = {"value": value, "unit": "solves*N/s", "cores": cores, "kind": "oracle",
            "sample": f"{desc}, Helmholtz + biharmonic per step, O(N) C oracle (Sec. 4 algorithms), float64"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves*N/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps * 1e3,
            "step": f"a bounded sample of the workload ({2 * rows} complex rows of {2 * full_rows})",
            "full_step_ms_extrapolated": 2 * full_rows / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, **w, "rows": full_rows,
                                            "sample_rows": rows},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "solves*N/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="n1024", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="auto",
                    help="fp64 | df for both problems; fp32_r1 | df_r1 for the Helmholtz problem (the "
                         "biharmonic one then in df); or auto (fastest path at the 1e-10 bar)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--streams", type=int, default=2, choices=[1, 2],
                    help="2 (default): the two independent solves on two forked streams, so that the second "
                         "kernel's blocks fill the SMs the first one's last round leaves idle; 1: in sequence")
    ap.add_argument("--graph", default="auto", choices=["auto", "on", "off"],
                    help="replay the step as a captured CUDA graph (auto: on for the batch workload)")
    ap.add_argument("--shard", action="store_true",
                    help="split the one field's modes into contiguous ranges, one per rank (shen_solve_modes); "
                         "strong scaling.  Default: one whole replica of the workload per rank (weak scaling)")
    ap.add_argument("--write-traffic", metavar="CSV", nargs="+",
                    help="rewrite profiles/traffic.json from ncu DRAM-bytes captures (one CSV per capture) on "
                         "--workload, then exit")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.write_traffic:
        print(json.dumps(write_traffic(args.write_traffic, w)["bytes_per_row"]))
        return
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    from paper_1701_03787_gb300 import Plan, inputs
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pci = gpu_pci_id(local)
    host_info = bind_gpu_local_host(pci) if pci else None
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    prec = resolve_precision(args.precision)
    # the large mixed workload (38.7 GB per field) runs lean: a plan with float-float
    # factors only, the two mean-flow Helmholtz solves at mode (0, 0) in the step, and
    # the end-to-end loop in place on two pinned host fields
    lean = args.workload in LEAN_WORKLOADS
    stream = torch.cuda.Stream()
    batched = args.workload == "batch"
    t_plan = time.perf_counter()
    if batched:
        from paper_1701_03787_gb300 import BatchPlan
        insts = inputs.batch_instances(w["n_inst"], seed=w["seed"])
        plan = BatchPlan(insts, stream=stream)
        N = None
        nm = plan.n_modes
        rows = plan.field_elems
    else:
        N = w["N"]
        plan = Plan(N, w["Nx"], w["Nz"], w["nu"], w["dt"], stream=stream, df_only=lean)
        nm = plan.n_modes
        rows = nm * N
    t_plan = time.perf_counter() - t_plan
    shard = args.shard and not batched and not lean
    m0, full_nm = 0, nm
    if shard:
        from paper_1701_03787_gb300.sharding import shard_range
        m0, nm = shard_range(full_nm, rank, world)
        rows = nm * N
    with torch.cuda.stream(stream):
        if shard:
            # this rank's columns of the one field (the same inputs on every rank count)
            f_h = inputs.rhs_torch(full_nm, N, seed=100)[m0:m0 + nm].clone()
            f_b = inputs.rhs_torch(full_nm, N, seed=200)[m0:m0 + nm].clone()
            torch.cuda.empty_cache()
        elif batched:
            f_h = inputs.batch_rhs_torch(plan.offsets, insts, seed=100 + rank)
            f_b = inputs.batch_rhs_torch(plan.offsets, insts, seed=200 + rank)
        else:
            f_h = inputs.rhs_torch(nm, N, seed=100 + rank)
            f_b = inputs.rhs_torch(nm, N, seed=200 + rank)
        u_h = torch.empty_like(f_h)
        u_b = torch.empty_like(f_b)
        if lean:
            f_m = inputs.rhs_torch(2, N, seed=300 + rank)       # mean-flow loads (two components)
            u_m = torch.empty_like(f_m)
    stream.synchronize()
    if batched:
        plan.helmholtz_solve = lambda f, u, precision, stream: plan.solve("helmholtz", f, u, precision, stream)
        plan.biharmonic_solve = lambda f, u, precision, stream: plan.solve("biharmonic", f, u, precision, stream)
    if shard:
        plan.helmholtz_solve = lambda f, u, precision, stream: plan.solve_modes("helmholtz", m0, f, u, precision,
                                                                                stream)
        plan.biharmonic_solve = lambda f, u, precision, stream: plan.solve_modes("biharmonic", m0, f, u,
                                                                                 precision, stream)
    tuned = None
    if args.precision == "auto" and not shard:
        # the library's autotuner times every path that meets the 1e-10 bar (and the
        # row-block shapes of the float-float kernels) on these fields and keeps the fastest
        tuned = {}
        for problem, f, u in (("helmholtz", f_h, u_h), ("biharmonic", f_b, u_b)):
            name, t = plan.autotune(problem, f, u, stream=stream)
            tuned[problem] = {"chosen": name, "ms": t}
            prec[problem] = name
        stream.synchronize()

    # The two solves are independent: run them on two streams that fork from and join
    # back into `stream`.  Each kernel's persistent grid fills every SM, so they overlap
    # only where the first one's last round of chains leaves SMs idle (N = 1024,
    # 1024 x 1024: 16.02 -> 15.76 ms per step).
    s_h, s_b = torch.cuda.Stream(), torch.cuda.Stream()
    fork, join_h, join_b = (torch.cuda.Event() for _ in range(3))

    def step(ph=prec["helmholtz"], pb=prec["biharmonic"]):
        if lean:                               # mean flow: Helmholtz at z = 0, mode 0 only
            plan.solve_modes("helmholtz", 0, f_m[0:1], u_m[0:1], precision=ph, stream=stream)
            plan.solve_modes("helmholtz", 0, f_m[1:2], u_m[1:2], precision=ph, stream=stream)
        if args.streams == 1:
            plan.helmholtz_solve(f_h, u_h, precision=ph, stream=stream)
            plan.biharmonic_solve(f_b, u_b, precision=pb, stream=stream)
            return
        fork.record(stream)
        s_h.wait_event(fork)
        s_b.wait_event(fork)
        plan.helmholtz_solve(f_h, u_h, precision=ph, stream=s_h)
        plan.biharmonic_solve(f_b, u_b, precision=pb, stream=s_b)
        join_h.record(s_h)
        join_b.record(s_b)
        stream.wait_event(join_h)
        stream.wait_event(join_b)

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    use_graph = args.graph == "on" or (args.graph == "auto" and batched)
    if use_graph:
        # the step's launches (and the batch queue resets) captured once, replayed per step
        graph = torch.cuda.CUDAGraph()
        eager_step = step
        with torch.cuda.graph(graph, stream=stream):
            eager_step()
        stream.synchronize()

        def step(ph=None, pb=None):
            if ph is not None or pb is not None:
                return eager_step(ph or prec["helmholtz"], pb or prec["biharmonic"])
            with torch.cuda.stream(stream):
                graph.replay()
        for _ in range(2):
            step()
        stream.synchronize()
    # timed region: K whole steps, CUDA events on `stream`
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(pci or local)
    clocks.start()
    time.sleep(0.5)                        # let nvidia-smi start before the timed region
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.mark_begin()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel durations, each kernel alone on `stream` (events on the launching stream)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for s in range(args.steps):
        ev[s][0].record(stream)
        plan.helmholtz_solve(f_h, u_h, precision=prec["helmholtz"], stream=stream)
        ev[s][1].record(stream)
        plan.biharmonic_solve(f_b, u_b, precision=prec["biharmonic"], stream=stream)
        ev[s][2].record(stream)
    torch.cuda.synchronize()
    t_h = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    t_b = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    # rhs_matvec (out = R x + beta y) for each problem, alone on `stream`: reads x and y,
    # writes out (48 algorithmic bytes per complex row)
    mv = None
    if not batched and not shard:
        out = torch.empty_like(f_h)
        pk, _ = peaks()
        mv = {"bytes_per_row": 48}
        for mprec in ("df", "fp64"):
            for _ in range(2):
                plan.rhs_matvec("helmholtz", u_h, y=f_h, beta=1.0, out=out, stream=stream, precision=mprec)
                plan.rhs_matvec("biharmonic", u_b, y=f_b, beta=1.0, out=out, stream=stream, precision=mprec)
            nrep = min(args.steps, 10)
            evm = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nrep)]
            for s in range(nrep):
                evm[s][0].record(stream)
                plan.rhs_matvec("helmholtz", u_h, y=f_h, beta=1.0, out=out, stream=stream, precision=mprec)
                evm[s][1].record(stream)
                plan.rhs_matvec("biharmonic", u_b, y=f_b, beta=1.0, out=out, stream=stream, precision=mprec)
                evm[s][2].record(stream)
            torch.cuda.synchronize()
            mh = float(np.mean([e[0].elapsed_time(e[1]) for e in evm]))
            mb = float(np.mean([e[1].elapsed_time(e[2]) for e in evm]))
            mv[mprec] = {"helmholtz_ms": mh, "biharmonic_ms": mb,
                         "frac_hbm": {"helmholtz": rows * 48 / (mh * 1e-3) / 1e9 / pk,
                                      "biharmonic": rows * 48 / (mb * 1e-3) / 1e9 / pk},
                         "traffic": {"helmholtz": measured_traffic(f"matvec_helmholtz:{mprec}", rows),
                                     "biharmonic": measured_traffic(f"matvec_biharmonic:{mprec}", rows)}}
        del out
    if not batched and not lean and not shard:
        # velocity recovery (f from u, then v and w): reads u, g, writes v, w (64 B per row)
        vv, ww = torch.empty_like(f_h), torch.empty_like(f_h)
        for _ in range(2):
            plan.velocity(u_b, u_h, vv, ww, stream=stream)
        nrep = min(args.steps, 10)
        ev_v = [torch.cuda.Event(enable_timing=True) for _ in range(nrep + 1)]
        for s in range(nrep):
            ev_v[s].record(stream)
            plan.velocity(u_b, u_h, vv, ww, stream=stream)
        ev_v[nrep].record(stream)
        torch.cuda.synchronize()
        mvel = float(np.mean([ev_v[s].elapsed_time(ev_v[s + 1]) for s in range(nrep)]))
        mv["velocity"] = {"ms": mvel, "bytes_per_row": 64, "frac_hbm": rows * 64 / (mvel * 1e-3) / 1e9 / pk,
                          "precision": "df", "traffic": measured_traffic("velocity:df", rows)}
        del vv, ww
        # the whole linear step (two operators, two solves, the velocity recovery): reads
        # u_old, g_old and both loads, writes u_new, g_new, v, w
        outs = tuple(torch.empty_like(f_h) for _ in range(4))
        for _ in range(2):
            plan.linear_step(f_b, f_h, u_b, u_h, out=outs, precision="auto", stream=stream)
        ev_l = [torch.cuda.Event(enable_timing=True) for _ in range(nrep + 1)]
        for s in range(nrep):
            ev_l[s].record(stream)
            plan.linear_step(f_b, f_h, u_b, u_h, out=outs, precision="auto", stream=stream)
        ev_l[nrep].record(stream)
        torch.cuda.synchronize()
        mls = float(np.mean([ev_l[s].elapsed_time(ev_l[s + 1]) for s in range(nrep)]))
        mv["linear_step"] = {"ms": mls, "value": rows * 2 / (mls * 1e-3), "unit": "solves*N/s",
                             "bytes_per_row": 128, "frac_hbm": rows * 128 / (mls * 1e-3) / 1e9 / pk}
        del outs
        if N & (N - 1) == 0:
            # wall-normal transforms of every mode column (Algorithms fst / ifst): read one
            # complex128 field, write one (32 algorithmic bytes per complex point)
            tr_out = torch.empty_like(f_h)
            trs = {"bytes_per_point": 32, "input": "the Helmholtz solution field"}
            for kind in ("inverse", "scalar", "forward"):
                for space in ("chebyshev", "dirichlet", "biharmonic"):
                    try:
                        for _ in range(2):
                            plan.transform(kind, space, u_h, out=tr_out, stream=stream)
                    except Exception as exc:             # a shape that does not fit this GPU
                        trs[f"{kind}_{space}"] = {"unsupported": str(exc)}
                        continue
                    ev_t = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
                    for s in range(5):
                        ev_t[s].record(stream)
                        plan.transform(kind, space, u_h, out=tr_out, stream=stream)
                    ev_t[5].record(stream)
                    torch.cuda.synchronize()
                    mt = float(np.mean([ev_t[s].elapsed_time(ev_t[s + 1]) for s in range(5)]))
                    trs[f"{kind}_{space}"] = {"ms": mt, "points_per_s": rows / (mt * 1e-3),
                                              "frac_hbm": rows * 32 / (mt * 1e-3) / 1e9 / pk,
                                              "traffic": measured_traffic(f"transform:{kind}_{space}", rows)}
            if rank == 0 and not args.no_cpu:
                trs["cpu_oracle"] = cpu_transforms(N)
            mv["transforms"] = trs
            del tr_out
    ms, = max_over_ranks([ms], pg, "cuda")
    step_rows = 2 * rows + (2 * N if lean else 0)            # complex rows solved per step
    # replicas: every rank solves the whole workload; shards: the ranks together solve it once
    value = (2 * full_nm * N if shard else world * step_rows) / (ms * 1e-3)

    # oracle-check samples, gathered now (later phases may reuse the device fields)
    sample = None
    if rank == 0 and not args.no_check and not batched:
        # (0, 0), the Nyquist modes and the corner (kx and kz Nyquist: the largest z2)
        special = [m for m in inputs.grid_modes(w["Nx"], w["Nz"]).values() if m0 <= m < m0 + nm]
        modes = [m + m0 for m in inputs.sample_modes(nm, 0.01 if nm * N <= 1e9 else 0.002, 3)]
        modes = sorted(set(modes) | set(special))
        refined = sorted(set(special) | set(modes[:: max(1, len(modes) // 48)]))
        idx = torch.as_tensor([m - m0 for m in modes], device="cuda")
        sample = (modes, refined, f_h[idx].cpu().numpy(), u_h[idx].cpu().numpy(),
                  f_b[idx].cpu().numpy(), u_b[idx].cpu().numpy())

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        def refill(h, t):                        # device -> pinned host, 256 MB copies
            hv, tv = h.view(-1), t.view(-1)
            for a0 in range(0, tv.numel(), 16 << 20):
                hv[a0:a0 + (16 << 20)].copy_(tv[a0:a0 + (16 << 20)], non_blocking=True)
            torch.cuda.synchronize()

        def pinned_copy(t):
            h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            refill(h, t)
            return h
        hf_h, hf_b = pinned_copy(f_h), pinned_copy(f_b)
        if lean:
            hu, hu2 = hf_h, hf_b                 # in place: each step solves the previous result
        else:
            hu = torch.empty_like(hf_h).pin_memory()
            hu2 = torch.empty_like(hf_b).pin_memory()

        if shard:
            def e2e_step():
                with torch.cuda.stream(stream):
                    f_h.copy_(hf_h, non_blocking=True)
                    f_b.copy_(hf_b, non_blocking=True)
                step()
                with torch.cuda.stream(stream):
                    hu.copy_(u_h, non_blocking=True)
                    hu2.copy_(u_b, non_blocking=True)
        else:
            # host fields straight into the library (shen_solve_host, shen_batch_solve_host):
            # chunked copy-in / solve / copy-out, the two solves issued on forked streams so
            # the pipeline runs through both
            def e2e_step():
                fork.record(stream)
                s_h.wait_event(fork)
                s_b.wait_event(fork)
                plan.solve_host("helmholtz", hf_h, hu, precision=prec["helmholtz"], stream=s_h)
                plan.solve_host("biharmonic", hf_b, hu2, precision=prec["biharmonic"], stream=s_b)
                join_h.record(s_h)
                join_b.record(s_b)
                stream.wait_event(join_h)
                stream.wait_event(join_b)
        # host link ceiling: plain copies of the same bytes in and out at once, 256 MB each
        def link_test():
            la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            # the copies are queued while the GPU sleeps, so the events time the copies and
            # not their submission from Python (which dominates small fields)
            with torch.cuda.stream(stream):
                torch.cuda._sleep(40_000_000)
            fork.record(stream)
            la.record(stream)
            s_h.wait_event(fork)
            s_b.wait_event(fork)
            ce = 16 << 20
            if lean:                             # H2D of one field while the other comes back
                pairs = ((f_h, hf_h, s_h), (hf_b, u_b, s_b))
            else:
                pairs = ((f_h, hf_h, s_h), (f_b, hf_b, s_h), (hu, u_h, s_b), (hu2, u_b, s_b))
            for dst, src, st in pairs:
                dv, sv = dst.view(-1), src.view(-1)
                with torch.cuda.stream(st):
                    for e0_ in range(0, dv.numel(), ce):
                        dv[e0_:e0_ + ce].copy_(sv[e0_:e0_ + ce], non_blocking=True)
            join_h.record(s_h)
            join_b.record(s_b)
            stream.wait_event(join_h)
            stream.wait_event(join_b)
            lb.record(stream)
            stream.synchronize()
            return sum(d.numel() for d, _, _ in pairs) * 16 / (la.elapsed_time(lb) * 1e-3) / 1e9

        link_before = [link_test() for _ in range(3)]
        e2e_step()
        stream.synchronize()
        # each step timed on its own; the median step is the figure (the host link is
        # shared with the machine's other jobs, which show up as outlying steps)
        k = max(3, min(args.steps, 9))
        ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        for i_ in range(k):
            ev_e[i_].record(stream)
            e2e_step()
        ev_e[k].record(stream)
        stream.synchronize()
        e2e_steps = [ev_e[i_].elapsed_time(ev_e[i_ + 1]) for i_ in range(k)]
        e2e_ms, = max_over_ranks([float(np.median(e2e_steps))], pg, "cuda")
        e2e = {"value": world * 2 * rows / (e2e_ms * 1e-3), "unit": "solves*N/s",
               "h2d_bytes_per_step": int(2 * rows * 16), "d2h_bytes_per_step": int(2 * rows * 16),
               "ms_per_step": e2e_ms, "ms_steps": e2e_steps, "timing": f"median of {k} steps",
               "path": ("device copies + solves" if shard else
                        "shen_batch_solve_host" if batched else "shen_solve_host"),
               "in_place": lean, "host": host_info}
        if not shard:
            # the host results must be the device path's bit for bit: fresh inputs in the
            # host buffers, one more step through the host path
            if lean:
                refill(hf_h, f_h)
                refill(hf_b, f_b)
            else:
                hu.zero_()
                hu2.zero_()
            e2e_step()
            stream.synchronize()
            pick = torch.as_tensor(np.linspace(0, hu.shape[0] - 1, 257).astype(np.int64))
            e2e["matches_device"] = bool(torch.equal(hu[pick], u_h[pick.cuda()].cpu())
                                         and torch.equal(hu2[pick], u_b[pick.cuda()].cpu()))
        link_after = [link_test() for _ in range(3)]
        link_gbs = max(link_before + link_after)
        e2e_gbs = 4 * rows * 16 / (e2e_ms * 1e-3) / 1e9
        e2e["roofline"] = {"bound": "host link (H2D + D2H concurrently)", "achieved": e2e_gbs, "peak": link_gbs,
                           "unit": "GB/s", "frac": e2e_gbs / link_gbs,
                           "peak_kind": "measured in this run: plain copies, both directions at once, queued "
                                        "before they start, the best of three passes before and three after "
                                        "the e2e steps",
                           "link_gbs_before_after": [link_before, link_after]}
        del hf_h, hf_b, hu, hu2

    # the float64 paths on the same fields, for the precision comparison: plain float64
    # sweeps and float64 sweeps + one double-double-residual refinement step (SHEN_FP64_R1)
    fp64_ms = None
    extra_samples = {}
    if not args.no_fp64_compare and not lean and (prec["helmholtz"] != "fp64" or prec["biharmonic"] != "fp64"):
        a, b, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        fp64_ms = {}
        paths = ("fp64",) if batched else ("fp64", "fp64_r1")
        for path in paths:
            for _ in range(2):
                step(path, path)
            a.record(stream)
            plan.helmholtz_solve(f_h, u_h, precision=path, stream=stream)
            b.record(stream)
            plan.biharmonic_solve(f_b, u_b, precision=path, stream=stream)
            c2.record(stream)
            stream.synchronize()
            key = "" if path == "fp64" else "_" + path
            fp64_ms["helmholtz" + key] = a.elapsed_time(b)
            fp64_ms["biharmonic" + key] = b.elapsed_time(c2)
            if sample is not None:
                extra_samples[path] = (u_h[idx].cpu().numpy(), u_b[idx].cpu().numpy())
        # float32 sweeps + refinement (shen_solve_refine, single-channel plans) for both
        # problems: one step with a float64 residual, two with a float-float one
        if not batched and not shard:
            work = torch.empty_like(f_h)
            for problem, fx, ux in (("helmholtz", f_h, u_h), ("biharmonic", f_b, u_b)):
                for steps, resid in ((1, "fp64"), (2, "df")):
                    plan.solve_refine(problem, fx, ux, work, steps=steps, residual=resid, stream=stream)
                    a.record(stream)
                    plan.solve_refine(problem, fx, ux, work, steps=steps, residual=resid, stream=stream)
                    b.record(stream)
                    stream.synchronize()
                    fp64_ms[f"{problem}_f32_r{steps}_{resid}"] = a.elapsed_time(b)
            del work
            # the fused float32-sweep + one-refinement-step kernels of the Helmholtz problem
            for name in ("df_r1", "fp32_r1"):
                try:
                    plan.helmholtz_solve(f_h, u_h, precision=name, stream=stream)
                except Exception:                    # not built for this N (limit of the fused kernels)
                    continue
                a.record(stream)
                plan.helmholtz_solve(f_h, u_h, precision=name, stream=stream)
                b.record(stream)
                stream.synchronize()
                fp64_ms[f"helmholtz_{name}"] = a.elapsed_time(b)
        step()                                   # leave the headline results in u_h, u_b
        stream.synchronize()

    velocity = mv.pop("velocity", None) if mv else None
    linear_step = mv.pop("linear_step", None) if mv else None
    transforms = mv.pop("transforms", None) if mv else None
    peak, peak_kind = peaks()
    dom = "biharmonic" if t_b >= t_h else "helmholtz"
    t_dom = max(t_b, t_h)
    achieved = rows * BYTES_PER_ROW / (t_dom * 1e-3) / 1e9
    traffic = None if batched else measured_traffic(f"{dom}:{prec[dom]}", rows)
    roofline = {"bound": "hbm", "kernel": f"solve_{dom}_{prec[dom]}", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "peak_kind": peak_kind, "bytes_per_row": BYTES_PER_ROW}
    line = {"metric": METRIC, "value": value, "unit": "solves*N/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong" if shard else "weak",
            "vs_baseline": None,
            "dtype": dtype_of(prec),
            "data": "synthetic", "precision": prec,
            "config": {"workload": args.workload, **w, "n_modes": nm, "n_classes": plan.n_classes, "rows": rows,
                       "streams": args.streams, "cuda_graph": use_graph, "plan_device_bytes": plan.info()[3]
                       if not batched else plan.device_bytes,
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"shard{world}" if shard else f"replicas{world}",
                       "mode_range": [m0, nm] if shard else None},
            "autotune": tuned, "kernel_ms": {"helmholtz": t_h, "biharmonic": t_b}, "compare_kernel_ms": fp64_ms, "plan_s": t_plan,
            "roofline": roofline, "gpu_launches": (4 if lean else 2) * args.steps, "clocks": clk, "e2e": e2e,
            "rhs_matvec": mv, "velocity": velocity, "linear_step": linear_step, "transforms": transforms}
    if sample is not None:
        modes, refined, F_h, U_h, F_b, U_b = sample
        head = "+".join(sorted(set(prec.values())))
        line["error_vs_oracle"] = oracle_errors(w, F_h, F_b, {head: (U_h, U_b), **extra_samples}, modes, refined)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_batch(w) if batched else cpu_baseline(w, args.precision)
    if rank == 0:
        print(json.dumps(line))
    plan.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
