"""The library's Fermi level (host code, Algorithm dc step 1) against the
oracle's bisection and closed forms; needs no GPU."""
import numpy as np
import pytest

from oracle import density as od


@pytest.fixture(scope="module")
def lib_fermi():
    from paper_1903_10959_gb300 import _lib
    try:
        _lib.load()
    except RuntimeError as e:
        pytest.skip(str(e))
    return _lib.fermi_level


@pytest.mark.parametrize("kT", [0.01, 0.05, 0.3])
@pytest.mark.parametrize("ne", [20.2, 23.0, 27.7])
def test_matches_oracle(lib_fermi, kT, ne):
    eps = np.array([-0.31, -0.2, -0.2, -0.05, 0.0, 0.12, 0.2, 0.33, 0.4])
    mu, occ = lib_fermi(eps, 6, ne, kT)
    mu_o, occ_o = od.fermi_level(eps, 6, ne, kT)
    assert abs(mu - mu_o) < 1e-12 * max(1.0, abs(mu_o)) + 1e-14
    assert np.allclose(occ, occ_o, atol=1e-12)
    assert abs(2 * (6 + occ.sum()) - ne) < 1e-11


def test_closed_form_and_errors(lib_fermi):
    from paper_1903_10959_gb300 import ChfsiError
    mu, occ = lib_fermi([0.0, 1.0], 0, 2.0, 0.25)
    assert abs(mu - 0.5) < 1e-13
    with pytest.raises(ChfsiError):
        lib_fermi([0.0, 1.0], 0, 4.5, 0.1)          # more electrons than states hold
