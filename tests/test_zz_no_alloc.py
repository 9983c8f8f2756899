"""The allocation-free Poisson entry point (for callers that cannot allocate device memory,
e.g. code recorded into a CUDA graph under a capture mode that forbids cudaMalloc, or a
framework that owns a fixed device pool) returns what the context-based poisson_field
returns, on two calls in a row that reuse its static scratch."""
import math

import numpy as np
import pytest
import torch

from paper_2606_29027_b300 import slar

pytestmark = pytest.mark.gpu


def _reference(N, L, rho):
    d = len(N)
    cfg = slar.make_config(dx=d, dv=d, N=tuple(N) + (8,) * d, lo=(0.0,) * (2 * d),
                           hi=tuple(L) + (1.0,) * d)
    ctx = slar.Context(cfg)
    E = torch.zeros((d, rho.numel()), dtype=torch.float64, device="cuda")
    phi = torch.zeros(rho.numel(), dtype=torch.float64, device="cuda")
    W = ctx.poisson_field(rho, E, phi)
    return E, phi, W


@pytest.mark.parametrize("N,L", [((64, 64), (4 * math.pi, 4 * math.pi)), ((128,), (10 * math.pi,)),
                                 ((32, 128), (3.0, 5.0))])
def test_static_poisson_matches_context_entry_point_twice(N, L):
    rng = np.random.default_rng(sum(N))
    for call in range(2):                       # second call reuses the same static scratch
        rho_h = rng.standard_normal(int(np.prod(N)))
        rho_h -= rho_h.mean()
        rho = torch.as_tensor(rho_h, device="cuda")
        E = torch.full((len(N), rho.numel()), float("nan"), dtype=torch.float64, device="cuda")
        phi = torch.full((rho.numel(),), float("nan"), dtype=torch.float64, device="cuda")
        W = slar.poisson_field_static(N, L, rho, E, phi)
        E_ref, phi_ref, W_ref = _reference(N, L, rho)
        torch.cuda.synchronize()
        assert torch.linalg.norm(E - E_ref) <= 1e-12 * torch.linalg.norm(E_ref)
        assert torch.linalg.norm(phi - phi_ref) <= 1e-12 * torch.linalg.norm(phi_ref)
        assert abs(W - W_ref) <= 1e-12 * W_ref


def test_static_poisson_rejects_oversize():
    rho = torch.zeros(256, dtype=torch.float64, device="cuda")
    E = torch.zeros(256, dtype=torch.float64, device="cuda")
    with pytest.raises(slar.SlarError):
        slar.poisson_field_static((256,), (1.0,), rho, E)
