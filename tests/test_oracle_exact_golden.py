"""Pin of the exact Riemann solver (used to pin the oracle's Sod run) against the
published star states of Toro (2009), Section 4.3.3, Table 4.3 (tests/golden)."""
import os

import numpy as np
import pytest

from oracle.exact import riemann_star, riemann_sample

GOLD = os.path.join(os.path.dirname(__file__), "golden", "toro_riemann_star.txt")


def _rows():
    out = []
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            out.append([float(v) for v in line.split()])
    return out


@pytest.mark.parametrize("row", _rows(), ids=lambda r: "test%d" % int(r[0]))
def test_star_state_matches_toro_table(row):
    _, rl, ul, pl, rr, ur, pr, ps, us, rsl, rsr = row
    g = 1.4
    p, u = riemann_star(rl, ul, pl, rr, ur, pr, g)
    assert p == pytest.approx(ps, rel=2e-4, abs=2e-5)
    assert u == pytest.approx(us, rel=2e-4, abs=2e-5)
    # densities just left and right of the contact
    eps = 1e-9
    r, _, _ = riemann_sample(rl, ul, pl, rr, ur, pr, g, np.array([u - eps, u + eps]))
    assert r[0] == pytest.approx(rsl, rel=2e-4, abs=2e-5)
    assert r[1] == pytest.approx(rsr, rel=2e-4, abs=2e-5)
