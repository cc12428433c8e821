"""The paper's second-order invariant of multiple-plane ray tracing (Sec. 2.1
and Sec. 5, Fig. 6): the E-mode shear power equals the convergence power and
the B-mode power equals the rotation power, B and omega being second order
in the potential.  On the sphere, with the final Jacobian of every ray shot
from a pixel centre taken in the basis at that pixel, both relations carry
the spin-2 factor s_l = (l + 2)(l - 1) / (l (l + 1)):
C_l^E = s_l C_l^kappa and C_l^B = s_l C_l^omega (for A the Jacobian of a map
of the sphere, E and kappa come from one scalar potential of the
displacement, B and omega from the other).

Workload: 8 independent lognormal planes (unit variance, C_l ~ l^-2,
band-limited at l = 48), shells of 250 Mpc/h to 2000 Mpc/h (flat LCDM,
Om = 0.25), source scale and growth per plane; rays at the 49152 pixel
centres of Nside 64, lens fields synthesised exactly at the rays (no map
interpolation), traced by the oracle's plane recursion and transport."""
import pytest
import torch

from oracle import healpix as hp, rays as orays, sht, spectra
from workloads import cosmology, synthetic

NSIDE, LP, NPLANES = 64, 48, 8


@pytest.fixture(scope="module")
def traced():
    pl = cosmology.lens_planes(NPLANES, 250.0)
    p = torch.arange(hp.npix(NSIDE))
    z, phi = hp.pix2ang_ring(NSIDE, p)
    lenses = []
    for m in range(NPLANES):
        modes = synthetic.random_field_modes(256, 2.0, LP, 1210003 + m)
        delta = synthetic.lognormal_density(z, phi, modes).double() - 1.0
        kappa = pl["scale"][m] * pl["growth"][m] * delta
        plm = sht.poisson(sht.analysis(kappa, NSIDE, LP), LP)
        lenses.append(lambda n, plm=plm: sht.lens_fields_at(plm, LP, n))
    n0 = hp.pix2vec_ring(NSIDE, p)
    st = orays.trace(n0, pl["chi"], lenses)
    nsrc = st["x"] / torch.linalg.vector_norm(st["x"], dim=-1, keepdim=True)
    return st["A"], orays.image_basis(st["A"], nsrc, n0)


def _band(S, lo, hi):
    l = torch.arange(LP + 1, dtype=torch.float64)
    s = torch.where(l >= 2, (l + 2) * (l - 1) / torch.where(l > 0, l * (l + 1), 1.0), torch.zeros_like(l))
    sel = (l >= lo) & (l <= hi)
    return S, s, sel


def test_b_mode_power_equals_rotation_power(traced):
    _, A = traced
    S = spectra.spectra_from_A(A, NSIDE, LP)
    S, s, sel = _band(S, 8, LP)
    ratio = float(S["B"][sel].sum() / (s[sel] * S["omega"][sel]).sum())
    assert abs(ratio - 1.0) < 0.01, ratio          # the paper: equal to about 1 %; here 0.08 %
    # both second order: far below E
    assert float(S["B"][sel].sum() / S["E"][sel].sum()) < 1e-3
    assert float(S["omega"][sel].sum()) > 0.0


def test_e_mode_power_equals_convergence_power(traced):
    _, A = traced
    S = spectra.spectra_from_A(A, NSIDE, LP)
    S, s, sel = _band(S, 2, LP)
    r = S["E"][sel] / (s[sel] * S["kappa"][sel])
    assert float((r - 1.0).abs().max()) < 5e-3, r    # largest deviation 0.19 %


def test_the_relation_needs_the_image_basis(traced):
    """With A left in the basis at the rays' source positions the shear is
    rotated by twice a first-order angle, which puts a second-order E
    component into B: the invariant then fails by a large factor."""
    A_src, _ = traced
    S = spectra.spectra_from_A(A_src, NSIDE, LP)
    S, s, sel = _band(S, 8, LP)
    ratio = float(S["B"][sel].sum() / (s[sel] * S["omega"][sel]).sum())
    assert ratio > 3.0, ratio
