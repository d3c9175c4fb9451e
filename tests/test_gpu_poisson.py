"""The particle-mesh Poisson solve (Section 3) on the GPU against the direct-summation
oracle of Eq. openbruteforceconv.

Tolerances: FP64 transforms |phi_gpu - phi_oracle| <= 1e-12 max|phi|: the FFT route rounds
each of its O(log2 N) butterfly stages in FP64 (about 1e-16 each), far below that bound.  FP32
transforms (MUSR_SPLIT): <= 2 log2(N) 2^-24 max|phi|, first-order rounding of the two
transforms' log2 N stages (N = 8 mx my mz, the doubled mesh); measured about 5 2^-24.  A wrong
index, spacing or normalisation is off by O(1).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _tol(B, prec, shape):
    return TOL if prec == B.MUSR_FP64 else 2.0 * np.log2(8.0 * np.prod(shape)) * 2.0 ** -24


@pytest.fixture(scope="module")
def B(musr_lib):
    from paper_1509_07685_gb300 import binding
    return binding


def _density(shape, seed, kind="random"):
    rng = np.random.default_rng(seed)
    if kind == "random":
        return rng.normal(size=shape)
    # a Gaussian bunch off the mesh centre (the beam of the paper's particle-mesh solver)
    axes = [np.arange(n) for n in shape]
    x, y, z = np.meshgrid(*axes, indexing="ij")
    c = [0.4 * n for n in shape]
    s = [0.12 * n + 0.5 for n in shape]
    return np.exp(-0.5 * (((x - c[0]) / s[0]) ** 2 + ((y - c[1]) / s[1]) ** 2 + ((z - c[2]) / s[2]) ** 2))


@pytest.mark.parametrize("shape,h", [((8, 8, 8), (1.0, 1.0, 1.0)), ((12, 10, 6), (0.3, 0.45, 0.2)),
                                     ((5, 1, 7), (0.7, 0.2, 1.3)), ((1, 1, 1), (0.5, 0.25, 2.0)),
                                     ((16, 9, 13), (0.05, 0.07, 0.11))])
@pytest.mark.parametrize("prec", [0, 1])
def test_poisson_matches_direct_sum(B, shape, h, prec):
    for kind, seed in (("random", 1), ("bunch", 2)):
        rho = _density(shape, seed, kind)
        ref = oracle.poisson_direct(rho, h)
        with B.Poisson(shape, h, prec) as ps:
            phi = ps.solve(rho)
            import torch
            d_rho = torch.tensor(rho, device="cuda")
            d_phi = torch.empty_like(d_rho)
            ps.solve_device(d_rho.data_ptr(), d_phi.data_ptr())
            torch.cuda.synchronize()
            phi_d = d_phi.cpu().numpy()
        assert np.max(np.abs(phi - ref)) <= _tol(B, prec, shape) * np.max(np.abs(ref)), (kind, np.max(np.abs(phi - ref)))
        assert np.array_equal(phi, phi_d)


@pytest.mark.parametrize("prec", [0, 1])
def test_poisson_sequence_of_densities(B, prec):
    """Solves of different densities in a row each match the oracle: the zero padding of the
    doubled mesh is written once and must survive the forward transform (out of place) and
    every later solve."""
    shape, h = (12, 10, 6), (0.3, 0.45, 0.2)
    point = np.zeros(shape)
    point[11, 0, 5] = 4.0
    seq = [_density(shape, 5, "random"), point, _density(shape, 6, "bunch"), _density(shape, 5, "random")]
    with B.Poisson(shape, h, prec) as ps:
        for rho in seq:
            ref = oracle.poisson_direct(rho, h)
            phi = ps.solve(rho)
            assert np.max(np.abs(phi - ref)) <= _tol(B, prec, shape) * np.max(np.abs(ref))


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 1])
def test_poisson_full_size_sampled(B, prec):
    """The paper's largest mesh (512 x 512 x 256, doubled to 1024 x 1024 x 512): sampled points
    against the oracle's direct sum at those points."""
    shape, h = (512, 512, 256), (0.01, 0.01, 0.02)
    rho = _density(shape, 3, "bunch")
    rng = np.random.default_rng(4)
    ijk = np.stack([rng.integers(0, n, 12) for n in shape], axis=1)
    ijk = np.vstack([ijk, [[0, 0, 0], [511, 511, 255], [204, 204, 102]]])
    ref = oracle.poisson_points(rho, h, ijk)
    with B.Poisson(shape, h, prec) as ps:
        ps.solve(np.random.default_rng(5).normal(size=shape))  # another density first
        phi = ps.solve(rho)
    got = phi[ijk[:, 0], ijk[:, 1], ijk[:, 2]]
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= _tol(B, prec, shape), err


def test_poisson_invalid_arguments(B):
    for shape, h in (((0, 4, 4), (1.0, 1.0, 1.0)), ((4, 4, 4), (1.0, -1.0, 1.0)), ((4, 4, 4), (1.0, np.nan, 1.0)),
                     ((1024, 1024, 1024), (1.0, 1.0, 1.0))):
        with pytest.raises(B.MusrError) as e:
            B.Poisson(shape, h)
        assert e.value.status == B.MUSR_EINVAL
    with pytest.raises(B.MusrError) as e:
        B.Poisson((4, 4, 4), (1.0, 1.0, 1.0), precision=7)
    assert e.value.status == B.MUSR_EINVAL
    with B.Poisson((4, 4, 4), (1.0, 1.0, 1.0)) as ps:
        with pytest.raises(ValueError):
            ps.solve(np.zeros((4, 4, 5)))
