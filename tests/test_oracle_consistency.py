"""Consistency of the oracle's numerical fluxes: with the same state on both sides of every
face the approximate Riemann flux must equal the physical flux (Section 2.3, Table 1
solvers): F(U, U) = F(U) for HLL, TVDLF and HLLC of every module."""
import numpy as np
import pytest

from oracle import Config, Solver

CASES = [("hd", "hll"), ("hd", "tvdlf"), ("hd", "hllc"), ("mhd", "hll"), ("mhd", "tvdlf"),
         ("srhd", "tvdlf"), ("ffhd", "tvdlf")]


def _state(physics, rng):
    if physics == "hd":
        return [rng.uniform(0.5, 2), *rng.normal(size=3), rng.uniform(0.5, 2)]
    if physics == "mhd":
        return [rng.uniform(0.5, 2), *rng.normal(size=3), rng.uniform(0.5, 2), *rng.normal(size=3), 0.1 * rng.normal()]
    if physics == "srhd":
        return [rng.uniform(0.5, 2), *(0.8 * rng.normal(size=3)), rng.uniform(0.1, 2)]
    b = rng.normal(size=3)
    return [rng.uniform(0.5, 2), rng.normal(), rng.uniform(0.5, 2), *(b / np.linalg.norm(b))]


@pytest.mark.parametrize("physics,flux", CASES)
def test_flux_of_equal_states_is_the_physical_flux(physics, flux):
    rng = np.random.default_rng(11)
    gamma = 4.0 / 3.0 if physics == "srhd" else 5.0 / 3.0
    s = Solver(Config(physics=physics, flux=flux, limiter="vanleer", gamma=gamma, base_blocks=(1, 1, 1)))
    ph = s.phys
    for _ in range(3):
        prim = np.array(_state(physics, rng), dtype=np.float64)
        P = np.broadcast_to(prim.reshape(-1, 1, 1, 1), (ph.nvar, 20, 20, 20)).copy()
        U = ph.prim2cons(prim.reshape(-1, 1))[:, 0]
        ch = 1.7
        for d in range(3):
            F = s._face_fluxes(P, d, s.dx(1), ch)
            if physics == "mhd":
                want = ph.flux(prim.reshape(-1, 1), U.reshape(-1, 1), d, ch)[:, 0]
            else:
                want = ph.flux(prim.reshape(-1, 1), U.reshape(-1, 1), d)[:, 0]
            got = F.reshape(ph.nvar, -1)
            scale = np.abs(want).max()
            assert np.max(np.abs(got - want[:, None])) <= 1e-14 * scale, (physics, flux, d)
