"""The float32 Euclidean select ranks L = (1 - g)(|q'|^2 + |r'|^2) - 2 q'.r'
(coordinates centred on a reference c, g = 4 (d + 6) 2^-24, clamped at 0), a
lower bound of the exact squared distance: references left out of a split are
then certified by the split's largest kept L.  These tests evaluate L in
float32 arithmetic (numpy, one rounding per operation, which bounds the
fused multiply-adds of the kernel as well) on inputs chosen to stress the
bound -- large offsets with and without centring, near duplicates, long rows --
and check it against the float64 distance.  No GPU."""
import numpy as np
import pytest

U = np.float32(2.0 ** -24)


def lower_bound_f32(Q, R, c):
    """L for every (query, reference) pair, in float32, as the select forms it."""
    d = Q.shape[1]
    g1 = np.float32(1.0) - np.float32(4.0) * np.float32(d + 6) * U
    q = (Q.astype(np.float32) - c.astype(np.float32)).astype(np.float32)
    r = (R.astype(np.float32) - c.astype(np.float32)).astype(np.float32)
    nq = np.zeros(q.shape[0], np.float32)
    nr = np.zeros(r.shape[0], np.float32)
    dot = np.zeros((q.shape[0], r.shape[0]), np.float32)
    for t in range(d):           # coordinate 0 first, one rounding per step
        nq = (nq + (q[:, t] * q[:, t]).astype(np.float32)).astype(np.float32)
        nr = (nr + (r[:, t] * r[:, t]).astype(np.float32)).astype(np.float32)
        dot = (dot + np.outer(q[:, t], r[:, t]).astype(np.float32)).astype(np.float32)
    s = (nq[:, None] + nr[None, :]).astype(np.float32)
    L = (g1 * s).astype(np.float32) - (np.float32(2.0) * dot).astype(np.float32)
    return np.maximum(L.astype(np.float32), np.float32(0.0))


def exact_sq(Q, R):
    q = Q.astype(np.float64)
    r = R.astype(np.float64)
    return ((q[:, None, :] - r[None, :, :]) ** 2).sum(-1)


@pytest.mark.parametrize("d", [3, 32, 96, 257])
@pytest.mark.parametrize("offset", [0.0, 1000.0, -3.5e4])
def test_lower_bound_never_exceeds_the_distance(d, offset):
    g = np.random.default_rng(1000 + d)
    R = (g.random((200, d)) + offset).astype(np.float32)
    Q = (g.random((40, d)) + offset).astype(np.float32)
    Q[:10] = R[:10]                                            # exact duplicates
    Q[10:20] = (R[10:20] + np.float32(1e-3) * g.standard_normal((10, d))).astype(np.float32)
    for c in (R[0], np.zeros(d, np.float32)):                   # centred, and not
        L = lower_bound_f32(Q, R, c)
        D = exact_sq(Q, R)
        assert np.all(L.astype(np.float64) <= D), np.max(L - D)


def test_centring_keeps_the_slack_at_the_scale_of_the_spread():
    """Far from the origin the uncentred bound loses everything (its slack
    exceeds the distances), while the centred one stays within a small
    fraction of them -- why the select centres its coordinates."""
    g = np.random.default_rng(7)
    d = 32
    R = (g.random((300, d)) + 1000.0).astype(np.float32)
    Q = (g.random((20, d)) + 1000.0).astype(np.float32)
    D = exact_sq(Q, R)
    L_far = lower_bound_f32(Q, R, np.zeros(d, np.float32))
    L_cen = lower_bound_f32(Q, R, R[0])
    assert np.all(L_far == 0.0)                                 # slack ~ 5e2 >> distances ~ 5
    gap = D - L_cen.astype(np.float64)
    assert np.all(gap >= 0.0) and np.max(gap / D) < 1e-4


def test_bound_is_tight_near_the_origin():
    """At the bench's scale (uniform [0, 1), d = 96) the slack is about
    g (|q|^2 + |r|^2), a few 1e-3 of the squared distances' size."""
    g = np.random.default_rng(11)
    d = 96
    R = g.random((150, d)).astype(np.float32)
    Q = g.random((30, d)).astype(np.float32)
    D = exact_sq(Q, R)
    L = lower_bound_f32(Q, R, R[0]).astype(np.float64)
    assert np.all(L <= D)
    assert np.max(D - L) < 2e-3
