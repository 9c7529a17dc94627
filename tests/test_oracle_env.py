"""Pins of the environment-prefiltering query generator (Sec. 5.4): the
compact-eps support property of the spherical Gaussian, its limits, the
paper's Q = 256 theta / pi, and the half-vector centre."""
import math

import numpy as np

import synth
from oracle import query as oq


def test_lobe_equals_eps_at_the_support_angle():
    A = np.array([0.5, 1.0, 3.0, 10.0])
    lam = np.array([2.0, 10.0, 50.0, 900.0])
    theta = oq.sg_support_angle(A, lam, 0.3)
    assert np.allclose(A * np.exp(lam * (np.cos(theta) - 1.0)), 0.3, rtol=1e-12)
    # inside the support the lobe is above eps, outside below
    assert np.all(A * np.exp(lam * (np.cos(0.9 * theta) - 1.0)) > 0.3)
    assert np.all(A * np.exp(lam * (np.cos(np.minimum(1.1 * theta, np.pi)) - 1.0)) < 0.3)


def test_support_limits():
    assert oq.sg_support_angle(np.array([0.3]), np.array([5.0]))[0] == 0.0     # A = eps
    assert oq.sg_support_angle(np.array([0.1]), np.array([5.0]))[0] == 0.0     # A < eps: nowhere
    assert oq.sg_support_angle(np.array([1e6]), np.array([0.1]))[0] == math.pi  # whole sphere


def test_square_side_and_centre():
    sg = np.zeros(1, dtype=synth.SG_DTYPE)
    sg["axis"] = [0.0, 0.0, 1.0]
    sg["amplitude"], sg["sharpness"] = 2.0, 20.0
    rec = np.zeros(1, dtype=synth.ENV_RECORD_DTYPE)
    rec["wo"] = [0.0, 0.0, 1.0]
    q = oq.env_queries(sg, rec, [256])
    theta = math.acos((math.log(0.3) - math.log(2.0)) / 20.0 + 1.0)
    Q = 256 * theta / math.pi  # Sec. 5.4 with a 256-pixel image
    assert np.isclose(q["s1"][0] - q["s0"][0], Q) and np.isclose(q["t1"][0] - q["t0"][0], Q)
    assert np.isclose((q["s0"][0] + q["s1"][0]) / 2, 128.0) and np.isclose((q["t0"][0] + q["t1"][0]) / 2, 128.0)
    # a tilted half vector moves the centre to its projected bin
    rec["wo"] = [math.sin(0.4), 0.0, math.cos(0.4)]
    q = oq.env_queries(sg, rec, [32])
    h = np.array([math.sin(0.4), 0.0, math.cos(0.4) + 1.0])
    h /= np.linalg.norm(h)
    assert np.isclose((q["s0"][0] + q["s1"][0]) / 2, (h[0] + 1) * 16)
