"""The wall-normal pipeline on the GPU against closed forms, with no oracle in the loop:
values of a right-hand side at the Gauss points -> scalar products (shen_transform,
Eq. sst1) -> Helmholtz or biharmonic solve (Sec. 4) -> inverse transform (Eq. ifft) ->
the exact solution at the points.

Manufactured solutions (the right-hand sides are their derivatives written out):
  Helmholtz   alpha u - u'' = g,  u = (1 - x^2) e^x, so
              u'' = -(1 + 4x + x^2) e^x and g = alpha u - u''  (u(+-1) = 0);
  biharmonic  u'''' + a u'' + b u = h,  u = p e^x with p = (1 - x^2)^2, so
              u'' = (p + 2p' + p'') e^x, u'''' = (p + 4p' + 6p'' + 4p''' + p'''') e^x
              (u(+-1) = u'(+-1) = 0),
with alpha = z2 + c, a = -(2 z2 + c), b = z2 (z2 + c), c = 2 / (nu dt) (the scaled systems
of the solves).  Both u are entire functions, so the Galerkin solutions converge
spectrally: at N = 64 the error at the points is at the level of rounding.
"""
import numpy as np
import pytest

from paper_1701_03787_gb300 import Plan

pytestmark = pytest.mark.gpu

NU, DT = 1 / 180, 1e-3
C = 2 / (NU * DT)
Z2 = np.array([0.0, 4.0, 37.0 ** 2, 1e4])
PHASE = 1.0 + 0.5j                       # complex columns: real and imaginary parts both exercised


def _points(N):
    return np.cos((2 * np.arange(N) + 1) * np.pi / (2 * N))


def _helmholtz(x, z2):
    ex = np.exp(x)
    u = (1 - x * x) * ex
    upp = -(1 + 4 * x + x * x) * ex
    return u, (z2 + C) * u - upp


def _biharmonic(x, z2):
    ex = np.exp(x)
    p = (1 - x * x) ** 2
    p1 = -4 * x + 4 * x ** 3
    p2 = -4 + 12 * x * x
    p3 = 24 * x
    p4 = 24.0
    u = p * ex
    u2 = (p + 2 * p1 + p2) * ex
    u4 = (p + 4 * p1 + 6 * p2 + 4 * p3 + p4) * ex
    a, b = -(2 * z2 + C), z2 * (z2 + C)
    return u, u4 + a * u2 + b * u


@pytest.mark.parametrize("precision", ["fp64", "df"])
@pytest.mark.parametrize("problem,space,rhs", [("helmholtz", "dirichlet", _helmholtz),
                                               ("biharmonic", "biharmonic", _biharmonic)])
@pytest.mark.parametrize("N", [64, 128])
def test_points_to_points(N, problem, space, rhs, precision):
    import torch
    x = _points(N)
    U = np.array([rhs(x, z)[0] for z in Z2]) * PHASE
    G = np.array([rhs(x, z)[1] for z in Z2]) * PHASE
    with Plan(N, z2=Z2, nu=NU, dt=DT) as plan:
        g = torch.as_tensor(G, device="cuda")
        f = plan.transform("scalar", space, g)                   # load vector (g, phi_k)_sigma
        coef = plan.solve(problem, f, precision=precision)
        u = plan.transform("inverse", space, coef).cpu().numpy()
    err = np.abs(u - U).max() / np.abs(U).max()
    assert err <= 1e-12, (N, problem, precision, err)
