"""Host check of the forward tensor-core theta kernel's ring assignment (theta_tc.cu,
tc_forward_body), restated here in Python: a launch of nrows rings with ncn polar-cap rings at
the front and ncs at the back runs on ntiles = ceil(nrows / 256) CTAs of 256 threads; the last wd
warps of every tile take the cap rings (then the plain rings the plain slots cannot hold), the
other warps the plain rings.  For every launch shape the samplings produce, each ring must be
owned by exactly one thread, and a cap ring only by a difference-form warp (the plain recurrence
is not accurate there).  The inverse tiles (64 rings from each end per 128-thread tile) are
checked the same way.
"""
import math

import numpy as np
import pytest


def forward_assignment(nrows, ncn, ncs, threads=256):
    ntiles = (nrows + threads - 1) // threads
    ncap = ncn + ncs
    wd = (ncap + 32 * ntiles - 1) // (32 * ntiles)
    dslots = 32 * wd
    pslots = threads - dslots
    nplain = nrows - ncap
    nplain_p = min(nplain, ntiles * pslots)
    owner = {}
    for tile in range(ntiles):
        for tid in range(threads):
            warp = tid // 32
            dform = warp >= threads // 32 - wd
            if dform:
                s = tile * dslots + (tid - pslots)
                act = s < ncap + (nplain - nplain_p)
                if s < ncn:
                    tr = s
                elif s < ncap:
                    tr = nrows - 1 - (s - ncn)
                else:
                    tr = ncn + nplain_p + (s - ncap)
            else:
                p = tile * pslots + tid
                act = p < nplain_p
                tr = ncn + p
            if act:
                assert 0 <= tr < nrows
                assert tr not in owner, (nrows, ncn, ncs, tr)
                owner[tr] = dform
    return owner, ntiles, wd


def inverse_assignment(nring, ring0=0, threads=128):
    nr = nring - ring0
    half = (nr + 1) // 2
    H = threads // 2
    ntiles = (half + H - 1) // H
    owner = {}
    for tile in range(ntiles):
        for tid in range(threads):
            q = tile * H + (tid % H)
            if tid < H:
                t = ring0 + q if q < half else -1
            else:
                t = nring - 1 - q if q < nr - half else -1
            if t >= 0:
                assert ring0 <= t < nring and t not in owner
                owner[t] = tile
    return owner


def caps(thetas):
    """Front / back counts of rings with sin(theta) < 0.15 (the difference form)."""
    diff = np.sin(thetas) < 0.15
    half = (len(thetas) + 1) // 2
    return int(diff[:half].sum()), int(diff[half:].sum()), diff


def sampling_rings(L, kind):
    if kind == "mw":
        t = np.arange(L)
        th = (2 * t + 1) * np.pi / (2 * L - 1)
        th[-1] = np.pi
        return th
    if kind == "mwss":                       # the interior rings run the recursion
        return np.pi * np.arange(1, L) / L
    return (2 * np.arange(2 * L) + 1) * np.pi / (4 * L)     # dh


@pytest.mark.parametrize("kind", ["mw", "mwss", "dh"])
@pytest.mark.parametrize("L", [2, 3, 17, 64, 130, 255, 256, 257, 511, 512, 1000, 1024])
def test_forward_rings_owned_once_and_caps_in_difference_warps(L, kind):
    th = sampling_rings(L, kind)
    nrows = len(th)
    if nrows == 0 or nrows > 2048:
        pytest.skip("no tensor-core forward launch")
    ncn, ncs, diff = caps(th)
    # the caps are contiguous at both ends
    assert diff[:ncn].all() and not diff[ncn:nrows - ncs].any() and diff[nrows - ncs:].all()
    owner, ntiles, wd = forward_assignment(nrows, ncn, ncs)
    assert sorted(owner) == list(range(nrows))
    assert ntiles <= 8 and wd <= 8
    for t, dform in owner.items():
        if diff[t]:
            assert dform


@pytest.mark.parametrize("L", [1536, 2047, 2048])
def test_forward_rings_at_the_largest_mw_launches(L):
    th = sampling_rings(L, "mw")
    ncn, ncs, diff = caps(th)
    owner, ntiles, wd = forward_assignment(len(th), ncn, ncs)
    assert sorted(owner) == list(range(len(th)))
    assert ntiles == math.ceil(L / 256) and wd == 1
    assert all(owner[t] for t in np.nonzero(diff)[0])


@pytest.mark.parametrize("nring,ring0", [(1, 0), (2, 0), (5, 0), (64, 0), (129, 0), (1023, 1), (1024, 0), (2048, 0)])
def test_inverse_tiles_cover_every_ring_once(nring, ring0):
    owner = inverse_assignment(nring, ring0)
    assert sorted(owner) == list(range(ring0, nring))
