"""Vortex diagnostics on analytic states with known winding (CPU)."""
import numpy as np
import pytest

from paper_2105_10517_gb300 import diagnostics, inputs


def vortex_state(n, charges, centres, length=12.0):
    x, y = inputs.grid(n, n, length, length)
    X, Y = np.meshgrid(x, y)
    psi = np.exp(-(X ** 2 + Y ** 2) / 8).astype(complex)
    for q, (a, b) in zip(charges, centres):
        z = (X - a) + 1j * np.sign(q) * (Y - b)
        psi = psi * z ** abs(q)
    return psi, x, y


@pytest.mark.parametrize("q", [-2, -1, 1, 2])
def test_central_winding_of_a_centred_vortex(q):
    psi, x, y = vortex_state(64, [q], [(0.0, 0.0)])
    assert diagnostics.central_winding(psi, x, y, 2.0) == q


def test_vortex_counts_of_a_lattice_piece():
    psi, x, y = vortex_state(96, [1, 1, -1], [(2.1, 0.3), (-1.7, 1.9), (0.2, -2.6)])
    stack = np.stack([psi, np.exp(-(x[None, :] ** 2 + y[:, None] ** 2)).astype(complex), np.conj(psi)])
    counts = diagnostics.vortex_counts(stack)
    assert counts[0] == (2, 1, 1)
    assert counts[1] == (0, 0, 0)
    assert counts[2] == (1, 2, -1)


def test_phase_noise_outside_the_condensate_is_not_counted():
    n = 64
    x, y = inputs.grid(n, n, 16.0, 16.0)
    X, Y = np.meshgrid(x, y)
    rho_amp = np.exp(-(X ** 2 + Y ** 2) / 2)
    rough = np.exp(1j * 2 * np.pi * inputs.uniform01(5, n * n).reshape(n, n))
    psi = np.where(X ** 2 + Y ** 2 > 49, 1e-9 * rough, rho_amp.astype(complex))
    assert diagnostics.vortex_counts(psi[None])[0] == (0, 0, 0)
