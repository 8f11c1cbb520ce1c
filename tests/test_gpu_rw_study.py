"""The synthetic analogue of Fig. 3: the adaptive-precision force error on the
defect atoms (CSP^list g > 1.5 A^2, the void's surface) against the precise
model evaluated on every atom, as a function of the averaging radius r_w of
Eq. 6 (Appendix B), float64 path, 27 511-atom void crystal.

The paper attributes the fall of the error with r_w to the defect atoms sitting
deeper inside the precise region, so that the fast model enters their forces
less.  Its two potentials are fitted to the same reference, so E^prec - E^EAM is
small in the bulk; the synthetic precise model (EAM + random ACE) is offset by a
constant dE^(0) = 0.72 eV per atom, and the grad-lambda force of Eq. 5 carries
that offset times grad lam.  With the models' energy zeros aligned
(prec_shift = dE^(0), which moves no force of either model) the test checks:

- the fast-model part of the error (the AP force without its grad-lambda term
  against the precise force) falls with r_w over 4-8 A, by an order of magnitude;
- the full AP error falls with it, and is then the fast-model part plus a
  grad-lambda part that stays small;
- without the alignment the grad-lambda part is the offset's, far larger;
- the selected atoms' energies are exact (they all have lam = 1)."""
import numpy as np
import pytest

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

RADII = [4.0, 5.0, 6.0, 7.0, 8.0]


@pytest.fixture(scope="module")
def rows():
    torch = torch_cuda()
    from paper_2512_07693_gb300 import rw_study
    return rw_study.study(torch, 24, RADII)["rows"]


def test_fast_model_error_falls_with_the_averaging_radius(rows):
    fast = [r["aligned_rmse_f_fast_model_part_ev_per_a"] for r in rows]
    assert all(b <= 1.05 * a for a, b in zip(fast, fast[1:])), fast
    assert fast[-1] < 0.1 * fast[0], fast
    # the force without the grad-lambda term does not depend on the energy zero
    np.testing.assert_allclose(fast, [r["rmse_f_fast_model_part_ev_per_a"] for r in rows], rtol=1e-9)


def test_ap_error_with_aligned_zeros_follows_the_fast_model_part(rows):
    tot = [r["aligned_rmse_f_ev_per_a"] for r in rows]
    assert all(b <= 1.05 * a for a, b in zip(tot, tot[1:])), tot
    assert tot[-1] < 0.1 * tot[0], tot
    for r in rows:
        assert r["aligned_rmse_f_grad_lambda_part_ev_per_a"] < 0.02, r
        assert r["rmse_f_grad_lambda_part_ev_per_a"] > 10 * r["aligned_rmse_f_grad_lambda_part_ev_per_a"], r
        assert r["atoms_selected"] > 100 and r["aligned_rmse_e_ev"] < 1e-9


def test_precise_fraction_grows_with_the_averaging_radius(rows):
    x = [r["x"] for r in rows]
    assert all(b > a for a, b in zip(x, x[1:])), x
