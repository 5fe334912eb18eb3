"""Pins of the naive FP64 oracle against facts fixed by the mathematics.

None of these re-types the oracle's loop: closed-form eigen-decays, FFT
convolution, conservation, exact fixed points and hand-derived steps.  The
pin-sensitivity tests at the end show that a transposed axis, a swapped offset
sign or a dropped term in the update would fail them.
"""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.golden import hand_steps

HEAT2D = [0.5, 0.125, 0.125, 0.125, 0.125]
JAC3D = [0.4] + [0.1] * 6
JAC1D = [1.0 / 3.0] * 3


def _fft_expected(u0, coeffs, T):
    """Periodic operator is a convolution: each Fourier coefficient is scaled
    by lambda(k) = sum_o c_o exp(+2 pi i k.o / n) per step (numpy's forward
    FFT uses exp(-2 pi i k x / n), so u[x+o] maps to exp(+2 pi i k o / n) U[k])."""
    d = u0.ndim
    n = u0.shape
    freqs = np.meshgrid(*[np.fft.fftfreq(m) * m for m in n], indexing="ij")
    lam = np.full(n, coeffs[0], dtype=np.complex128)
    k = 1
    for a in range(d):
        for o in (-1, 1):
            lam = lam + coeffs[k] * np.exp(2j * np.pi * freqs[a] * o / n[a])
            k += 1
    return np.real(np.fft.ifftn(np.fft.fftn(u0) * lam ** T))


@pytest.mark.parametrize("sizes,T,seed", [((11,), 5, 1), ((7, 5), 4, 2), ((5, 6, 4), 3, 3)])
def test_fft_convolution_asymmetric(oracle_lib, sizes, T, seed):
    c = si.random_coefficients(len(sizes), 1, seed)
    u0 = si.uniform_grid(sizes, seed + 10, periodic=True)
    got = oracle.sweep(u0, sizes, c, T, periodic=True)
    exp = _fft_expected(u0, c, T)
    scale = np.sum(np.abs(c)) ** T
    assert np.max(np.abs(got - exp)) <= 1e-12 * scale


@pytest.mark.parametrize("sizes,coeffs,T", [((64,), JAC1D, 40), ((24, 20), HEAT2D, 30), ((12, 10, 8), JAC3D, 16)])
def test_fourier_mode_decay(oracle_lib, sizes, coeffs, T):
    """cos mode of wave vector k decays by lambda(k) = c0 + 2 sum_a c1 cos(2 pi k_a / n_a)."""
    u0, (amps, ks, phases) = si.fourier_grid(sizes, seed=3)
    got = oracle.sweep(u0, sizes, coeffs, T, periodic=True)
    d = len(sizes)
    axes = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in sizes], indexing="ij", sparse=True)
    exp = np.zeros(sizes)
    for m in range(len(amps)):
        lam = coeffs[0] + 2.0 * sum(coeffs[1 + 2 * a] * math.cos(2 * math.pi * ks[m, a] / sizes[a]) for a in range(d))
        arg = phases[m] + sum(2 * math.pi * ks[m, a] * axes[a] / sizes[a] for a in range(d))
        exp = exp + amps[m] * lam ** T * np.cos(arg)
    assert np.max(np.abs(got - exp)) <= 1e-12 * float(np.sum(amps))


@pytest.mark.parametrize("sizes,coeffs,modes,T", [((15,), [0.5, 0.25, 0.25], (3,), 9),
                                                  ((9, 13), HEAT2D, (2, 5), 12),
                                                  ((6, 7, 5), JAC3D, (1, 2, 3), 7)])
def test_dirichlet_sine_mode(oracle_lib, sizes, coeffs, modes, T):
    """With a zero ring, prod_a sin(p_a pi j_a / (n_a + 1)) (j_a = 1..n_a) decays
    by c0 + 2 c1 sum_a cos(p_a pi / (n_a + 1)) per step."""
    d = len(sizes)
    shape = tuple(n + 2 for n in sizes)
    g = np.ones(shape)
    for a in range(d):
        j = np.arange(shape[a], dtype=np.float64)
        s = np.sin(modes[a] * np.pi * j / (sizes[a] + 1))
        s[0] = 0.0
        s[-1] = 0.0
        g = g * s.reshape([-1 if b == a else 1 for b in range(d)])
    lam = coeffs[0] + 2 * coeffs[1] * sum(math.cos(modes[a] * math.pi / (sizes[a] + 1)) for a in range(d))
    got = oracle.sweep(g, sizes, coeffs, T)
    assert np.max(np.abs(got - lam ** T * g)) <= 1e-13


def test_sum_conserved_periodic(oracle_lib):
    sizes, T = (17, 13), 25
    u0 = si.uniform_grid(sizes, 7, periodic=True)
    got = oracle.sweep(u0, sizes, HEAT2D, T, periodic=True)
    s0 = oracle.grid_sum(u0, sizes, periodic=True)
    s1 = oracle.grid_sum(got, sizes, periodic=True)
    bound = T * 5 * 2.0 ** -53 * float(np.sum(np.abs(u0))) * 4
    assert abs(s1 - s0) <= bound


def test_constant_field_exact(oracle_lib):
    """Heat-2D weights are dyadic: a dyadic constant is reproduced bitwise."""
    sizes = (9, 11)
    g = np.full(sizes, 0.75)
    got = oracle.sweep(g, sizes, HEAT2D, 13, periodic=True)
    assert np.array_equal(got, g)
    z = np.zeros((11, 13))
    assert np.array_equal(oracle.sweep(z, sizes, HEAT2D, 5), z)


def test_linear_profile_fixed_point(oracle_lib):
    """Jacobi-1D with weights 1/3: the line through the two ring values is a fixed point."""
    n = 30
    a, b = 0.25, 1.75
    g = a + (b - a) * np.arange(n + 2) / (n + 1)
    got = oracle.sweep(g, (n,), JAC1D, 50)
    assert np.max(np.abs(got - g)) <= 1e-13


@pytest.mark.parametrize("case", hand_steps(), ids=lambda c: c["name"])
def test_hand_derived_steps(oracle_lib, case):
    got = oracle.sweep(case["init"], case["sizes"], case["coeffs"], case["T"], periodic=case["periodic"])
    assert np.array_equal(got, case["expected"])


def test_ring_untouched_and_threads_bitwise(oracle_lib):
    sizes = (13, 7, 9)
    g = si.uniform_grid(sizes, 5, ring="random")
    a = oracle.sweep(g, sizes, JAC3D, 6, threads=1)
    b = oracle.sweep(g, sizes, JAC3D, 6, threads=4)
    assert np.array_equal(a, b)
    mask = np.ones(g.shape, dtype=bool)
    mask[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(a[mask], g[mask])


def test_T_zero_is_identity(oracle_lib):
    g = si.uniform_grid((5, 5), 9)
    assert np.array_equal(oracle.sweep(g, (5, 5), HEAT2D, 0), g)


# ---- pin sensitivity: plausible mistakes fail the pins above -------------

def test_pin_detects_swapped_offset_sign(oracle_lib):
    sizes, T = (7, 5), 3
    c = si.random_coefficients(2, 1, 2)
    u0 = si.uniform_grid(sizes, 12, periodic=True)
    swapped = c.copy()
    swapped[[1, 2]] = swapped[[2, 1]]          # axis-0 -1 and +1 exchanged
    bad = oracle.sweep(u0, sizes, swapped, T, periodic=True)
    assert np.max(np.abs(bad - _fft_expected(u0, c, T))) > 1e-6


def test_pin_detects_transposed_axes(oracle_lib):
    sizes, T = (7, 5), 3
    c = si.random_coefficients(2, 1, 4)
    u0 = si.uniform_grid(sizes, 13, periodic=True)
    transposed = c[[0, 3, 4, 1, 2]]
    bad = oracle.sweep(u0, sizes, transposed, T, periodic=True)
    assert np.max(np.abs(bad - _fft_expected(u0, c, T))) > 1e-6


def test_pin_detects_dropped_term(oracle_lib):
    sizes, T = (24, 20), 10
    u0, (amps, ks, phases) = si.fourier_grid(sizes, seed=3)
    dropped = list(HEAT2D)
    dropped[4] = 0.0
    bad = oracle.sweep(u0, sizes, dropped, T, periodic=True)
    good = oracle.sweep(u0, sizes, HEAT2D, T, periodic=True)
    assert np.max(np.abs(bad - good)) > 1e-3


def test_max_rel_error_definition():
    ref = np.array([1.0, -4.0, 2.0])
    u = np.array([1.0, -4.0 + 2e-5, 2.0])
    assert oracle.max_rel_error(u, ref) == pytest.approx(2e-5 / 4.0)


def test_pointwise_rel_error_definition():
    """Hand-computed cases of the floored pointwise error: a cell's own
    magnitude divides its difference; cells below 1e-3 of the maximum use
    that floor instead."""
    ref = np.array([4.0, 0.5, 1e-6, -2.0])
    u = ref + np.array([0.0, 1e-6, 2e-9, -4e-6])
    # per cell: 0/4, 1e-6/0.5, 2e-9/max(1e-6, 4e-3), 4e-6/2
    assert oracle.pointwise_rel_error(u, ref) == pytest.approx(2e-6)
    # a wrong small cell that the normwise measure does not see
    bad = ref.copy()
    bad[1] += 2e-5
    assert oracle.max_rel_error(bad, ref) == pytest.approx(5e-6)
    assert oracle.pointwise_rel_error(bad, ref) == pytest.approx(4e-5)
    # below the floor: the floor divides
    tiny = ref.copy()
    tiny[2] += 4e-8
    assert oracle.pointwise_rel_error(tiny, ref) == pytest.approx(1e-5)
    e = oracle.errors(u, ref)
    assert e["normwise"] == pytest.approx(1e-6) and e["pointwise"] == pytest.approx(2e-6)
    assert oracle.pointwise_rel_error(np.zeros(3), np.zeros(3)) == 0.0
