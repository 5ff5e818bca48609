"""The transverse spin estimator of honeycomb_check.spin_structure_factors against its zz
counterpart and the oracle: at U = 0 (free fermions, SU(2) exact at any dtau) S_xx equals
S_zz, and S_zz equals the oracle's own structure factor on the same configuration."""
import numpy as np

from oracle import dqmc
from oracle.dqmc import Chain, Model
from paper_2106_00712_gb300.honeycomb_check import spin_structure_factors
from paper_2106_00712_gb300.workloads import random_fields


def _gtilde(model, G):
    P = dqmc.Propagators(model)
    return P.expK_ph @ G @ P.expK_mh


def test_free_fermions_give_equal_zz_and_xx():
    model = Model(3, 2, 1.0, 0.0, 2.0, 0.1, 5, seed=1, lattice="honeycomb")
    ch = Chain(model, random_fields(1, model.L_tau, model.N, seed=3)[0], 0)
    gu, gd = (_gtilde(model, G) for G in ch.G)
    p = dqmc.staggered_signs(model.Lx, model.Ly, model.lattice)
    zz, xx = spin_structure_factors(gu, gd, p)
    assert abs(zz - xx) < 1e-12 * abs(zz)


def test_zz_matches_the_oracle_estimator_on_an_interacting_configuration():
    model = Model(3, 2, 1.0, 4.0, 2.0, 0.1, 5, seed=2, lattice="honeycomb")
    ch = Chain(model, random_fields(1, model.L_tau, model.N, seed=4)[0], 0)
    P = dqmc.Propagators(model)
    want = dqmc.measure(P, model, ch.G[0], ch.G[1])["s_pipi"]
    gu, gd = (_gtilde(model, G) for G in ch.G)
    p = dqmc.staggered_signs(model.Lx, model.Ly, model.lattice)
    zz, xx = spin_structure_factors(gu, gd, p)
    assert abs(zz - want) < 1e-12 * abs(want)
    assert xx != zz   # the HS field breaks SU(2) configuration by configuration
