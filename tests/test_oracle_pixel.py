"""Pins of the oracle's pixelised parity channel (Sec. 3.2: spoke directions
quantised to one pixel byte per edge, degenerate tetrahedra with |V| < 1e-9
excluded from the odd channel).

The paper leaves the pixel scheme open; the reading here is 256 equal-area
pixels (16 bands of equal width in cos(theta) times 16 sectors of equal
width in phi). The pins: the pixel of integer directions against an
independent high-precision restatement (mpmath) on random, tiny and
edge-straddling directions; pixel volumes against high precision; the gap
between degenerate and non-degenerate pixel volumes over every ordered pixel
triple (so that rounding can never move a tetrahedron across the 1e-9
threshold); the whole channel against all-tuples brute force; the paper's
injection test; the even channel unchanged; a tetrahedron whose two spokes
share a pixel excluded from the odd channel.
"""
import itertools
import json
import os

import numpy as np
import pytest

import catalogs
import oracle
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def special_directions():
    out = []
    for v in itertools.product((-2, -1, 0, 1, 2), repeat=3):
        if any(v):
            out.append(v)
    # near the sector edge at tan(pi/8) = 0.41421...: 5/12 above, 41/99 below
    for a, b in ((12, 5), (99, 41), (70, 29), (169, 70), (408, 169)):
        for sx, sy in itertools.product((1, -1), repeat=2):
            out += [(sx * a, sy * b, 3), (sx * b, sy * a, -7), (sx * a, sy * b, 0)]
    # near band edges of cos(theta): z / |d| close to k/8 - 1
    for k in range(1, 16):
        t = k / 8 - 1
        for r in (1000, 30000, 400000):
            z = int(round(t * r))
            for x in (r, r + 1):
                y = int(round(np.sqrt(max(r * r - z * z - 0, 0)))) if x == r else 0
                out.append((y, 0, z))
                out.append((7, y, z))
    return np.array(out, dtype=np.int64)


def test_direction_pixels_match_independent_reference():
    rng = np.random.default_rng(5)
    d = np.concatenate([special_directions(),
                        rng.integers(-40000, 40001, size=(3000, 3)),
                        rng.integers(-5, 6, size=(500, 3))])
    d = d[np.any(d != 0, axis=1)]
    got = oracle.direction_pixels(d)
    ref = np.array([bf.direction_pixel(*v) for v in d.tolist()], dtype=np.uint8)
    assert np.array_equal(got, ref)
    # every pixel is reached, and the 16 x 16 layout holds
    dense = rng.normal(size=(200_000, 3)) * 1e5
    pix = oracle.direction_pixels(np.round(dense).astype(np.int64))
    assert len(np.unique(pix)) == 256


def test_pixels_have_equal_area():
    """Uniform directions fill the 256 pixels equally (chi-square)."""
    rng = np.random.default_rng(6)
    v = rng.normal(size=(512_000, 3))
    v = np.round(v / np.linalg.norm(v, axis=1)[:, None] * 1e6).astype(np.int64)
    counts = np.bincount(oracle.direction_pixels(v), minlength=256)
    expect = len(v) / 256
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 255 + 6 * np.sqrt(2 * 255)


def test_pixel_volumes_match_high_precision():
    import mpmath
    mpmath.mp.dps = 40
    rng = np.random.default_rng(7)
    trip = rng.integers(0, 256, size=(400, 3))
    got = oracle.pixel_volumes(trip)

    def centre(p):
        band, sector = divmod(int(p), 16)
        zc = mpmath.mpf(-1) + (band + mpmath.mpf(1) / 2) / 8
        phi = (sector + mpmath.mpf(1) / 2) * mpmath.pi / 8
        rho = mpmath.sqrt(1 - zc * zc)
        return [rho * mpmath.cos(phi), rho * mpmath.sin(phi), zc]

    for (p1, p2, p3), g in zip(trip.tolist(), got):
        a, b, c = centre(p1), centre(p2), centre(p3)
        v = (a[1] * b[2] - a[2] * b[1]) * c[0] + (a[2] * b[0] - a[0] * b[2]) * c[1] + \
            (a[0] * b[1] - a[1] * b[0]) * c[2]
        assert abs(float(v) - g) < 1e-15


def test_pixel_volume_gap_over_every_triple():
    """Over all 256^3 ordered pixel triples the FP64 pixel volume is either
    below 1e-14 in magnitude (mathematically zero: repeated pixels or three
    pixels on one great circle) or above 5e-5, so no evaluation order or
    last-bit difference can move a tetrahedron across the 1e-9 threshold,
    and the sign is the same in every evaluation order."""
    p = np.arange(256)
    band, sector = p // 16, p % 16
    zc = -1.0 + (band + 0.5) / 8.0
    phi = (sector + 0.5) * np.pi / 8.0
    rho = np.sqrt(1.0 - zc * zc)
    u = np.stack([rho * np.cos(phi), rho * np.sin(phi), zc], axis=1)
    cross = np.cross(u[:, None, :], u[None, :, :])           # [256, 256, 3]
    V = np.einsum("ijk,lk->ijl", cross, u)                    # V[i, j, l]
    a = np.abs(V)
    assert a[a < 1e-9].max() < 1e-14
    assert a[a >= 1e-9].min() > 5e-5
    # the oracle's own evaluation agrees in sign and degeneracy
    rng = np.random.default_rng(8)
    trip = rng.integers(0, 256, size=(20000, 3))
    got = oracle.pixel_volumes(trip)
    ref = V[trip[:, 0], trip[:, 1], trip[:, 2]]
    assert np.array_equal(np.abs(got) >= 1e-9, np.abs(ref) >= 1e-9)
    assert np.array_equal(np.sign(got[np.abs(got) >= 1e-9]), np.sign(ref[np.abs(ref) >= 1e-9]))


@pytest.mark.parametrize("periodic,seed", [(True, 31), (False, 32), (True, 33)])
def test_pixel_parity_matches_bruteforce(periodic, seed):
    box_u = 20_000
    edges_u = np.array([0, 1800, 3000, 4200], dtype=np.int64)
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.integers(0, box_u, size=(50, 3)),
                        np.mod(10_000 + rng.integers(-2600, 2601, size=(30, 3)), box_u)])
    X = X.astype(np.int32)
    bu = box_u if periodic else 0
    e_ref, o_ref = bf.count4_pixel(X, bu, edges_u)
    assert e_ref.sum() > 30 and np.abs(o_ref).sum() > 0
    e, o = oracle.Graph(X, bu, edges_u, nthreads=2).count_4pcf(pixel=True)
    assert np.array_equal(e, e_ref) and np.array_equal(o, o_ref)


@pytest.mark.parametrize("mirrored_fraction", [0.0, 0.3, 0.5])
def test_pixel_parity_injection(mirrored_fraction):
    """Sec. 4.9 with pixelised directions: the injected shape is far from
    degenerate, so every copy, whatever its rotation and vertex order, keeps
    its handedness: odd = N_L - N_R exactly."""
    with open(os.path.join(GOLDEN, "injection_tetrahedron.json")) as f:
        gold = json.load(f)
    edges_u = np.array(gold["edges_u"], dtype=np.int64)
    n = gold["n_struct"]
    _, lat, mirrored = catalogs.lattice_tetrahedra(np.array(gold["shape_u"]), n, mirrored_fraction,
                                                   gold["box_u"], int(edges_u[-1]) + 1, seed=78)
    g = oracle.Graph(lat.astype(np.int32), gold["box_u"], edges_u)
    even, odd = g.count_4pcf(pixel=True)
    k = [oracle.config_bins(4, len(edges_u) - 1, i)[0]
         for i in range(oracle.num_configs(4, len(edges_u) - 1))].index(tuple(gold["rep"]))
    n_left, n_right = int((~mirrored).sum()), int(mirrored.sum())
    assert even[k] == n and even.sum() == n
    assert odd[k] == gold["left_sign"] * (n_left - n_right)
    e_exact, o_exact = g.count_4pcf()
    assert np.array_equal(even, e_exact) and np.array_equal(odd, o_exact)


def test_pixel_even_channel_and_weights():
    box_u = 30_000
    edges_u = np.array([0, 2000, 3500, 5000], dtype=np.int64)
    rng = np.random.default_rng(9)
    X = np.mod(15_000 + rng.integers(-4000, 4001, size=(300, 3)), box_u).astype(np.int32)
    w = catalogs.uniform_weights(len(X), seed=10)
    g = oracle.Graph(X, box_u, edges_u)
    e, o, we, wo = g.count_4pcf(w, pixel=True)
    ex, ox, wex, wox = g.count_4pcf(w)
    assert np.array_equal(e, ex) and np.array_equal(we, wex)
    e1, o1, _, wo1 = g.count_4pcf(np.ones(len(X), np.float32), pixel=True)
    assert np.array_equal(wo1, o1.astype(np.float64)) and np.array_equal(o1, o)


def test_spokes_in_one_pixel_are_degenerate():
    """A thin chiral tetrahedron whose spokes from the origin (its smallest
    index) to the second and third vertex fall in the same pixel has an exact
    V != 0 but a pixel volume of zero: the exact channel counts it, the
    pixelised channel does not."""
    P = np.array([[0, 0, 0], [3000, 1200, 400], [3100, 1210, 380], [200, 2600, 1500]])
    pix = oracle.direction_pixels(P[1:] - P[0])
    assert pix[0] == pix[1] != pix[2]
    box_u = 100_000
    X = (P + 20_000).astype(np.int32)
    # the six edges (102.5, 3009, 3256, 3318, 3349, 3405) each in their own
    # bin: all bins distinct, so the configuration is chiral
    edges_u = np.array([0, 1000, 3100, 3300, 3330, 3380, 3450], dtype=np.int64)
    g = oracle.Graph(X, box_u, edges_u)
    e, o = g.count_4pcf()
    ep, op = g.count_4pcf(pixel=True)
    assert e.sum() == 1 and np.array_equal(e, ep)
    k = int(np.argmax(e))
    assert oracle.config_bins(4, 6, k)[1], "the configuration must be chiral"
    assert abs(int(o[k])) == 1 and op[k] == 0
