"""Pins of the oracle's J2 plasticity (the history-dependent matrix law of
Example 1, Sec. 5.1) and of its hyper-reduced evaluation with history:
closed forms and identities the mechanics fix."""
import numpy as np
import pytest

import synthetic as syn
from synthetic import meshes
from conftest import rom_path
from oracle import cluster, j2, law, macro, reduced

E_M = 1.0
MU, KA = law.mu_kappa_from_E_nu(E_M, 0.3)
LAM = KA - 2.0 * MU / 3.0
SY0, HK = 0.01 * E_M, 0.016 * E_M            # Example 1: sigma_y0 = 0.01 E, h = 0.016 E


def _eps(e11, e22, e12):
    e = np.zeros((3, 3))
    e[0, 0], e[1, 1], e[0, 1], e[1, 0] = e11, e22, e12, e12
    return e


def test_elastic_range_is_hooke():
    eps = _eps(1e-3, -4e-4, 6e-4)
    h0 = np.zeros(7)
    sig, C, h1 = j2.return_map(eps, h0, MU, KA, SY0, HK)
    assert np.abs(sig - (LAM * np.trace(eps) * np.eye(3) + 2 * MU * eps)).max() < 1e-15
    assert np.array_equal(h1, h0)


def test_pure_shear_closed_form():
    # proportional shear eps_12 = gamma / 2: the flow direction is fixed, so
    # |eps_p| = (2 mu |e| - sqrt(2/3) sy0) / (2 mu + 2 h / 3) with |e| = gamma / sqrt2,
    # tau = |s| / sqrt2, whatever the number of increments
    gamma = 0.05
    ne = gamma / np.sqrt(2.0)
    epn = (2 * MU * ne - np.sqrt(2.0 / 3.0) * SY0) / (2 * MU + 2 * HK / 3)
    tau = 2 * MU * (ne - epn) / np.sqrt(2.0)
    for steps in (1, 7):
        h = np.zeros(7)
        for k in range(1, steps + 1):
            sig, C, h = j2.return_map(_eps(0, 0, gamma * k / steps / 2), h, MU, KA, SY0, HK)
        assert abs(sig[0, 1] - tau) <= 1e-14
        assert abs(h[6] - np.sqrt(2.0 / 3.0) * epn) <= 1e-14


def test_return_lands_on_the_yield_surface_and_is_isochoric():
    g = syn.rng(syn.SEED_BASE + 290)
    for _ in range(20):
        e = g.standard_normal(3) * 0.02
        h0 = np.zeros(7)
        h0[:6] = g.standard_normal(6) * 1e-3
        h0[2] = -(h0[0] + h0[1])
        h0[4:6] = 0.0
        h0[6] = abs(g.standard_normal()) * 1e-3
        sig, C, h1 = j2.return_map(_eps(*e), h0, MU, KA, SY0, HK)
        s = sig - np.trace(sig) / 3 * np.eye(3)
        if h1[6] > h0[6]:
            assert abs(np.sqrt(np.sum(s * s)) - np.sqrt(2 / 3) * (SY0 + HK * h1[6])) <= 1e-14
            assert abs(h1[0] + h1[1] + h1[2]) <= 1e-16


@pytest.mark.parametrize('plastic', [False, True])
def test_consistent_tangent_is_the_derivative_of_the_return_map(plastic):
    g = syn.rng(syn.SEED_BASE + 291)
    scale = 0.02 if plastic else 1e-3
    for _ in range(5):
        e = g.standard_normal(3) * scale
        eps = _eps(*e)
        sig, C, h1 = j2.return_map(eps, np.zeros(7), MU, KA, SY0, HK)
        assert (h1[6] > 0) == plastic
        hh = 1e-7
        for k in range(3):
            for l in range(3):
                de = np.zeros((3, 3))
                de[k, l] += 0.5 * hh
                de[l, k] += 0.5 * hh
                sp, _, _ = j2.return_map(eps + de, np.zeros(7), MU, KA, SY0, HK)
                sm, _, _ = j2.return_map(eps - de, np.zeros(7), MU, KA, SY0, HK)
                fd = (sp - sm) / (2 * hh)
                an = 0.5 * (C[:, :, k, l] + C[:, :, l, k])
                assert np.abs(fd - an).max() <= 1e-7 * np.abs(C).max()


def test_elastic_unloading_leaves_the_plastic_stress():
    # load into the plastic range, unload to zero strain: the stress is
    # -2 mu eps_p (elastic unloading from the stored history)
    # (shear 30% beyond first yield: the reverse trial stays inside the surface)
    h = np.zeros(7)
    _, _, h = j2.return_map(_eps(0.0, 0.0, 0.01), h, MU, KA, SY0, HK)
    assert h[6] > 0.0
    sig, _, h2 = j2.return_map(np.zeros((3, 3)), h, MU, KA, SY0, HK)
    ep = np.zeros((3, 3))
    for k, (i, jj) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        ep[i, jj] = ep[jj, i] = h[k]
    assert np.abs(sig + 2 * MU * ep).max() <= 1e-15 and np.array_equal(h2, h)


def test_elastic_rom_with_history_law_is_linear_and_matches_the_hyperelastic_tangent():
    # with an infinite yield stress the J2 ROM is the small-strain linear
    # ROM: its converged stress is linear in U - I, and its tangent at I is
    # the Neo-Hooke ROM's tangent at I (both laws linearize to Hooke)
    orom = reduced.Rom.load(rom_path('c1'))
    plastic = np.array([[np.inf, 0.0], [np.inf, 0.0]])
    C0 = cluster.initial_stiffness(orom)
    H = np.array([[2e-4, -1e-4], [-1e-4, 3e-4]])
    out = []
    for s_ in (1.0, 2.0):
        st = reduced.zero_state(orom)
        st['Uprev'] = np.array([1.0, 1.0, 0.0])
        hist = np.zeros((orom.m, 7))
        for _ in range(4):
            o = j2.eval_point(orom, plastic, np.eye(2) + s_ * H, hist=hist, **st)
            st = dict(q=o['q'], s=o['s'], S=o['S'], Uprev=o['Uprev'])
        out.append(o)
    assert out[0]['rnorm'] < 1e-14
    assert np.abs(out[1]['Palg'] - 2 * out[0]['Palg']).max() <= 1e-12 * np.abs(out[0]['Palg']).max()
    # at U = I + H the linear ROM's Pbar_U equals C0 : H
    assert np.abs(out[0]['Palg'].ravel() - C0 @ H.ravel()).max() <= 1e-10 * np.abs(C0 @ H.ravel()).max()


def test_load_unload_is_irreversible():
    # uniaxial tension of a 2x2 Q4 square to 2% strain and back to zero:
    # with the plastic matrix the reaction at zero displacement is not zero
    # (plastic strain remains), with an elastic matrix it is
    orom = reduced.Rom.load(rom_path('c1'))
    X, conn = meshes.rect(2, 2)
    prob = macro.uniaxial_problem(macro.MacroMesh(X, conn), 0.02)
    lf = [0.5, 1.0, 0.8, 0.6, 0.4, 0.2, 0.0]      # unloading in small steps (monolithic predictor)
    plastic = np.array([[SY0, HK], [np.inf, 0.0]])
    res = j2.driver(prob, orom, plastic, lf)
    ela = j2.driver(prob, orom, np.array([[np.inf, 0.0], [np.inf, 0.0]]), lf)
    assert abs(ela['reactions'][-1]) <= 1e-10 * abs(ela['reactions'][1])
    assert abs(res['reactions'][-1]) > 1e-2 * abs(res['reactions'][1])
    assert res['reactions'][1] < ela['reactions'][1]             # softer once yielded
    assert res['hist'][..., 6].max() > 0.0
