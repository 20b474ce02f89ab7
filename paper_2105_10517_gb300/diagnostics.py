"""Host-side diagnostics of a fetched wave function (not part of the time step).

Vortex count: a vortex of component c sits in a grid plaquette when the phase
of psi_c winds by +-2 pi around the plaquette's four corners (the sum of the
wrapped phase differences along its edges).  Only plaquettes inside the
condensate are counted -- some grid point within `halo` points of the
plaquette has rho_c > rel_density max(rho_c) -- so phase noise in the empty
outskirts does not count, while vortex cores (where rho_c itself vanishes) do.
"""
import numpy as np
from scipy.ndimage import maximum_filter


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def winding_map(psi_c):
    """Integer winding number of every plaquette (shape (ny-1, nx-1))."""
    ph = np.angle(psi_c)
    d1 = _wrap(ph[:-1, 1:] - ph[:-1, :-1])   # (j, i) -> (j, i+1)
    d2 = _wrap(ph[1:, 1:] - ph[:-1, 1:])     # (j, i+1) -> (j+1, i+1)
    d3 = _wrap(ph[1:, :-1] - ph[1:, 1:])     # (j+1, i+1) -> (j+1, i)
    d4 = _wrap(ph[:-1, :-1] - ph[1:, :-1])   # (j+1, i) -> (j, i)
    return np.rint((d1 + d2 + d3 + d4) / (2 * np.pi)).astype(int)


def vortex_counts(psi, rel_density=1e-3, halo=3):
    """Per component: (number of vortices, number of antivortices, net winding)."""
    out = []
    for c in range(psi.shape[0]):
        rho = np.abs(psi[c]) ** 2
        w = winding_map(psi[c])
        near = maximum_filter(rho, size=2 * halo + 1, mode="constant")
        ok = near[:-1, :-1] > rel_density * rho.max()
        w = np.where(ok, w, 0)
        out.append((int(np.sum(w > 0)), int(np.sum(w < 0)), int(np.sum(w))))
    return out


def central_winding(psi_c, x, y, radius):
    """Winding of the phase of psi_c along the square ring of the grid cells at
    distance ~radius from the origin (counter-clockwise)."""
    ny, nx = psi_c.shape
    ic = int(np.argmin(np.abs(x))), int(np.argmin(np.abs(y)))
    h = max(1, int(round(radius / (x[1] - x[0]))))
    i0, i1 = max(ic[0] - h, 0), min(ic[0] + h, nx - 1)
    j0, j1 = max(ic[1] - h, 0), min(ic[1] + h, ny - 1)
    path = [(j0, i) for i in range(i0, i1)] + [(j, i1) for j in range(j0, j1)] + \
           [(j1, i) for i in range(i1, i0, -1)] + [(j, i0) for j in range(j1, j0, -1)]
    ph = np.array([np.angle(psi_c[j, i]) for j, i in path])
    return int(np.rint(np.sum(_wrap(np.diff(np.append(ph, ph[0])))) / (2 * np.pi)))
