"""Tensor-core split-precision recurrence product (tcgen05 + TMA) against float64 references.

fo_recurrence_product computes out = alpha A B^T + beta C + D + shift I with the operands
split into 16-bit planes. References are float64 torch products:
* BF16x1: the bf16-rounded operands multiplied exactly; the kernel differs only by float32
  accumulation, relative Frobenius error <= 1e-5;
* BF16x3: the float32 operands multiplied exactly, relative error <= 2e-6 (float32 level);
* FP16x2: entries scaled into the fp16 range, relative error <= 2e-5.
Sizes cover one tile, several tiles and a ragged edge (n not a multiple of 128).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

TOL = {"bf16x1": 1e-5, "bf16x3": 1e-6, "fp16x2": 2e-6}


def rand(n, seed, sym=False):
    g = torch.Generator(device="cpu").manual_seed(seed)
    a = (torch.rand((n, n), generator=g, dtype=torch.float64) * 2 - 1) / math.sqrt(n)
    if sym:
        a = 0.5 * (a + a.T)
    return a.float().to(DEV)


def ref_product(a, b, prec):
    if prec == "bf16x1":
        return a.bfloat16().double() @ b.bfloat16().double().T
    return a.double() @ b.double().T


def relerr(x, ref):
    return float((x.double() - ref).norm() / ref.norm())


@pytest.mark.parametrize("prec", ["bf16x1", "bf16x3", "fp16x2"])
@pytest.mark.parametrize("n", [128, 200, 256, 384, 1000, 2048])
def test_full_product(solver, prec, n):
    a, b = rand(n, 1), rand(n, 2)
    out = solver.recurrence_product(a, b, precision=prec, symmetric=False)
    torch.cuda.synchronize()
    assert relerr(out, ref_product(a, b, prec)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x1", "bf16x3", "fp16x2"])
@pytest.mark.parametrize("n", [128, 300, 1000])
def test_symmetric_product_is_exactly_symmetric(solver, prec, n):
    # A and B commuting symmetric matrices (polynomials of one symmetric S): A B is symmetric
    s = rand(n, 7, sym=True)
    a = s
    b = (s.double() @ s.double()).float() * 0.5
    b = 0.5 * (b + b.T)
    out = solver.recurrence_product(a, b, precision=prec, symmetric=True)
    torch.cuda.synchronize()
    assert torch.equal(out, out.T)
    # the upper triangle is computed; for BF16x1 the rounded operands no longer commute,
    # so only that triangle is compared with the product of the rounded operands
    ref = ref_product(a, b, prec)
    iu = torch.triu_indices(n, n, device=DEV)
    ou, ru = out.double()[iu[0], iu[1]], ref[iu[0], iu[1]]
    assert float((ou - ru).norm() / ru.norm()) <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x1"])
def test_recurrence_epilogue(solver, prec):
    n = 300
    a, b, c, d = rand(n, 3, True), rand(n, 4, True), rand(n, 5), rand(n, 6)
    out = solver.recurrence_product(a, b, c, d, alpha=2.0, beta=-1.0, shift=-1.0, precision=prec,
                                    symmetric=False)
    ref = 2.0 * ref_product(a, b, prec) - c.double() + d.double() - torch.eye(n, dtype=torch.float64, device=DEV)
    assert relerr(out, ref) <= TOL[prec] * 4


def test_product_of_chebyshev_matrices_bf16x3(solver):
    # T_2 = 2 X X - I for a scaled tight-binding Hamiltonian
    n = 512
    h = synth.tight_binding(n, 9)
    ea, eb = O.gershgorin_bounds(h)
    x = O.scale_hamiltonian(h, ea, eb)
    xt = torch.from_numpy(x).float().to(DEV)
    t2 = solver.recurrence_product(xt, xt, alpha=2.0, shift=-1.0, precision="bf16x3",
                                   symmetric=True)
    ref = torch.from_numpy(2 * x @ x - np.eye(n)).to(DEV)
    assert float((t2.double() - ref).abs().max()) <= 1e-6
    assert torch.equal(t2, t2.T)
