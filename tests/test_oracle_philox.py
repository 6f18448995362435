"""Pins of the oracle's Philox-4x32-10 generator and its uniform conversion."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_vectors():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        vals = [int(x, 16) for x in f[1:]]
        rows.append((vals[0:4], vals[4:6], vals[6:10]))
    return rows


def test_philox_known_answer_vectors(oracle):
    rows = kat_vectors()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        assert oracle.philox4x32_10(ctr, key) == expect


def test_ray_uniforms_are_top_23_bits_plus_half(oracle):
    for seed, rid in [(1, 0), (4, 12345), (2**40 + 7, 2**33 + 5)]:
        ctr = [rid & 0xffffffff, rid >> 32, 0, 0]
        key = [seed & 0xffffffff, seed >> 32]
        w = oracle.philox4x32_10(ctr, key)
        a, b = oracle.ray_uniforms(seed, rid)
        assert a == ((w[0] >> 9) + 0.5) / 2**23
        assert b == ((w[1] >> 9) + 0.5) / 2**23
        assert 0.0 < a < 1.0 and 0.0 < b < 1.0


def test_ray_uniforms_are_uniform(oracle):
    xs = np.array([oracle.ray_uniforms(9, i) for i in range(20000)])
    # mean 1/2 and variance 1/12 within a few standard errors
    assert abs(xs.mean() - 0.5) < 0.01
    assert abs(xs.var() - 1.0 / 12.0) < 0.005
    assert abs(np.corrcoef(xs[:, 0], xs[:, 1])[0, 1]) < 0.03
