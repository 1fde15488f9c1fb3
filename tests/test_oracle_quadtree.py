"""Pins of the oracle's quadtree partition (Sec. 6.2, RA-Quadtree).

* lookup: the leaf returned for a state is the one whose rectangle, rebuilt
  independently from the tree's structure, contains (u0, u1);
* refinement: one pass equals a literal transcription of the rule -- every
  leaf with more than M_split visits since the previous pass splits once into
  four children that inherit lambda and n / 4 (at least 1);
* stationarity: after refinement stops changing the tree, the visits of the
  leaves follow their closed-form masses (App. B with uneven regions).
"""
import math

import numpy as np

from paper_2402_08273_gb300 import scenes as S

TOY = S.TOY_DEFAULT


def _chains(oracle_mod, **kw):
    args = dict(n_chains=128, width=64, height=64, region_px=8, max_depth=0, epoch_len=16,
                n_bootstrap=1 << 12, p_large=0.2, partition=1, qt_max_leaves=256, qt_max_depth=6,
                qt_split=600, qt_refine=128 * 16 * 4)
    args.update(kw)
    ch = oracle_mod.Chains(oracle_mod.Scene(toy=TOY), **args)
    ch.init()
    return ch


def _rects(child, leaf):
    """leaf id -> [x0, x1, y0, y1] from the structure alone (root = [0,1)^2,
    child j covers the quadrant with bit x = j & 1, bit y = j >> 1)."""
    out = {}

    def walk(n, x0, x1, y0, y1):
        if child[n][0] < 0:
            out[int(leaf[n])] = (x0, x1, y0, y1)
            return
        xm, ym = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
        for j in range(4):
            walk(child[n][j], xm if j & 1 else x0, x1 if j & 1 else xm, ym if j >> 1 else y0, y1 if j >> 1 else ym)

    walk(0, 0.0, 1.0, 0.0, 1.0)
    return out


def test_quadtree_lookup_matches_rectangles(oracle_mod):
    ch = _chains(oracle_mod)
    ch.run_epochs(40)
    child, leaf, depth = ch.quadtree()
    assert ch.n_regions > 16
    rects = _rects(child, leaf)
    assert sorted(rects) == list(range(ch.n_regions))
    area = sum((r[1] - r[0]) * (r[3] - r[2]) for r in rects.values())
    assert area == 1.0                                      # leaves tile the screen
    rng = np.random.default_rng(2)
    for _ in range(5000):
        q = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
        u0, u1 = q[0] / 2.0 ** 32, q[1] / 2.0 ** 32
        x0, x1, y0, y1 = rects[ch.region_of(q)]
        assert x0 <= u0 < x1 and y0 <= u1 < y1


def test_refinement_pass_matches_rule(oracle_mod):
    split = 1500
    ch = _chains(oracle_mod, qt_split=split, qt_refine=10 ** 12)   # passes only when asked
    ch.run_epochs(6)
    for _ in range(4):
        child0, leaf0, depth0 = (a.copy() for a in ch.quadtree())
        h0 = ch.hist.astype(np.int64).copy()
        lam0, n0 = ch.lam.copy(), ch.n_updates.copy()
        # visits since the previous pass (h minus its snapshot at that pass)
        hp0 = h0 - ch.hist_since_pass.astype(np.int64)
        m0 = ch.n_regions
        ch.refine()
        child1, leaf1, depth1 = ch.quadtree()
        # literal transcription: leaves in node order, > split visits -> four children
        expect_split = [n for n in range(len(child0)) if child0[n][0] < 0 and h0[leaf0[n]] - hp0[leaf0[n]] > split
                        and depth0[n] < 6]
        m = m0
        for n in range(len(child0)):
            if n in expect_split:
                k = leaf0[n]
                assert child1[n][0] >= 0 and leaf1[n] == -1
                ids = [leaf1[child1[n][j]] for j in range(4)]
                assert ids[0] == k and ids[1:] == [m, m + 1, m + 2]
                m += 3
                for j in range(4):
                    assert depth1[child1[n][j]] == depth0[n] + 1
                    assert child1[child1[n][j]][0] < 0                # not split again in this pass
                for i in ids:
                    assert ch.lam[i] == lam0[k]
                    assert ch.n_updates[i] == max(1, n0[k] // 4)
                    assert ch.visits[i] == 0 and ch.accsum[i] == 0 and ch.hist[i] == 0
            else:
                assert (child1[n] == child0[n]).all() and leaf1[n] == leaf0[n]
        assert ch.n_regions == m
        ch.run_epochs(3)


def test_quadtree_histogram_follows_leaf_mass(oracle_mod):
    ch = _chains(oracle_mod, n_chains=256, qt_split=3000, qt_refine=256 * 16 * 10, qt_max_leaves=64)
    ch.run_epochs(200)            # refinement stops at 64 leaves
    child, leaf, depth = ch.quadtree()
    assert ch.n_regions >= 61
    rects = _rects(child, leaf)
    mass = np.array([S.toy_rect_mass(TOY, *rects[k]) for k in range(ch.n_regions)])
    ch.run_epochs(1)             # ensure a pass boundary is behind us
    base = ch.hist.astype(np.float64).copy()
    ch.run_epochs(100)
    child2, _, _ = ch.quadtree()
    assert len(child2) == len(child)                        # no further splits
    v = ch.hist.astype(np.float64) - base
    tv = 0.5 * np.abs(v / v.sum() - mass / mass.sum()).sum()
    assert tv < 0.03, tv
