"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds no arithmetic of the method: it only draws right-hand sides and lists
modes.  Load vectors follow the workload recipe: entry j of every column is
(X_j + i Y_j) / (1 + j)^2 with X, Y ~ N(0, 1) i.i.d.
"""
import numpy as np


def spectrum(N):
    return 1.0 / (1.0 + np.arange(N)) ** 2


def rhs_numpy(n_modes, N, seed):
    """complex128 (n_modes, N) from numpy's PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((n_modes, N))
    y = rng.standard_normal((n_modes, N))
    return (x + 1j * y) * spectrum(N)[None, :]


def rhs_torch(n_modes, N, seed, device="cuda", chunk_modes=65536):
    """complex128 (n_modes, N) drawn on `device` with torch's generator (large fields)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((n_modes, N), dtype=torch.complex128, device=device)
    w = torch.as_tensor(spectrum(N), device=device)
    for m0 in range(0, n_modes, chunk_modes):
        m1 = min(n_modes, m0 + chunk_modes)
        re = torch.randn((m1 - m0, N), generator=g, device=device, dtype=torch.float64)
        im = torch.randn((m1 - m0, N), generator=g, device=device, dtype=torch.float64)
        out[m0:m1] = torch.complex(re * w, im * w)
    return out


def sample_modes(n_modes, fraction, seed, must_include=()):
    """Sorted seeded sample of mode indices (without replacement) plus `must_include`."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    k = max(1, int(round(fraction * n_modes)))
    picks = set(rng.choice(n_modes, size=min(k, n_modes), replace=False).tolist())
    picks.update(int(m) for m in must_include if 0 <= m < n_modes)
    return sorted(picks)


def grid_modes(Nx, Nz):
    """Named modes of a (Nx/2+1) x Nz mode-major grid: (0,0), the Nyquists, the corner."""
    nxh = Nx // 2 + 1
    return {"mean": 0, "kz_nyquist": Nz // 2, "kx_nyquist": (nxh - 1) * Nz,
            "corner": (nxh - 1) * Nz + Nz // 2, "last": nxh * Nz - 1}


def batch_instances(n_inst, seed, Ns=(64, 96, 128, 256, 512), grids=(16, 32, 64),
                    nu_range=(1e-4, 1e-2), dt_range=(1e-4, 1e-2)):
    """Instance list of the batching workload: N uniform over Ns, Nx and Nz i.i.d. uniform
    over grids, nu log-uniform and dt uniform over the given ranges (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    out = []
    for _ in range(n_inst):
        out.append({"N": int(rng.choice(Ns)), "Nx": int(rng.choice(grids)), "Nz": int(rng.choice(grids)),
                    "nu": float(np.exp(rng.uniform(np.log(nu_range[0]), np.log(nu_range[1])))),
                    "dt": float(rng.uniform(dt_range[0], dt_range[1]))})
    return out


def batch_rhs_torch(offsets, instances, seed, device="cuda"):
    """Batched field (flat complex128) with each instance's block drawn as rhs_torch."""
    import torch
    out = torch.empty(offsets[-1], dtype=torch.complex128, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    for i, inst in enumerate(instances):
        N = inst["N"]
        n = (offsets[i + 1] - offsets[i]) // N
        w = torch.as_tensor(spectrum(N), device=device)
        re = torch.randn((n, N), generator=g, device=device, dtype=torch.float64) * w
        im = torch.randn((n, N), generator=g, device=device, dtype=torch.float64) * w
        out[offsets[i]:offsets[i + 1]] = torch.complex(re, im).reshape(-1)
    return out
