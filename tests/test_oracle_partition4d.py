"""Oracle pins for the 4-D partition in primary sample space: the region of a
state is its screen region crossed with a dir_cells x dir_cells grid over the
first bounce's BSDF coordinates (u5, u6).

- the lookup against the index written out from its definition;
- pointwise detailed balance of the state-dependent Kelemen kernel across
  4-D regions of different sigma, with an independently written density
  (every dimension's offset must lie in the reverse kernel's support);
- chain invariants on the Cornell box (histogram total, region count).
"""
import math

import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S


def _chains(oracle_mod, g=3, **kw):
    sc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    args = dict(n_chains=32, width=64, height=64, region_px=32, max_depth=3, epoch_len=8, n_bootstrap=1 << 12,
                dir_cells=g)
    args.update(kw)
    return oracle_mod.Chains(sc, **args)


def test_lookup_matches_definition(oracle_mod):
    g = 3
    ch = _chains(oracle_mod, g)
    assert ch.m == 4 * g * g
    rng = np.random.default_rng(0)
    for _ in range(2000):
        q = rng.integers(0, 2 ** 32, ch.D, dtype=np.uint64).astype(np.uint32)
        px = ((int(q[0]) >> 8) * 64) >> 24
        py = ((int(q[1]) >> 8) * 64) >> 24
        cu = ((int(q[5]) >> 8) * g) >> 24
        cv = ((int(q[6]) >> 8) * g) >> 24
        assert ch.region_of(q) == ((px // 32) + (py // 32) * 2) * g * g + cu + cv * g


def test_needs_grid_plain_scene(oracle_mod):
    with pytest.raises(ValueError):
        _chains(oracle_mod, 2, target_mode=1)
    with pytest.raises(ValueError):
        oracle_mod.Chains(oracle_mod.Scene(toy=S.TOY_DEFAULT), n_chains=8, max_depth=0, dir_cells=2)


def _kelemen_density(delta, sigma, s1, s2):
    a = np.abs(delta)
    inside = (a >= sigma * s1) & (a <= sigma * s2)
    return np.where(inside, 0.5 / (a * math.log(s2 / s1)), 0.0).prod()


def test_detailed_balance_across_4d_regions(oracle_mod):
    ch = _chains(oracle_mod, 2, max_depth=1)
    rng = np.random.default_rng(4)
    sig = rng.uniform(0.6, 2.5, ch.m).astype(np.float32)
    ch.sigma[:] = sig
    sc = ch.scene
    s1, s2 = 1 / 1024, 1 / 64
    D = ch.D
    checked = across = 0
    for _ in range(4000):
        x = rng.integers(0, 2 ** 32, D, dtype=np.uint64).astype(np.uint32)
        kx = ch.region_of(x)
        sx = float(sig[kx])
        mag = np.exp(rng.uniform(math.log(sx * s1), math.log(sx * s2), D))
        dq = np.rint(rng.choice([-1, 1], D) * mag * 2 ** 32).astype(np.int64)
        y = ((x.astype(np.int64) + dq) % 2 ** 32).astype(np.uint32)
        ky = ch.region_of(y)
        sy = float(sig[ky])
        delta = dq / 2 ** 32
        rel = np.concatenate([np.abs(np.abs(delta) / (s * b) - 1) for s in (sx, sy) for b in (s1, s2)])
        if rel.min() < 1e-5:
            continue
        fx = sc.path_eval(x, 64, 64, 1)[0]
        fy = sc.path_eval(y, 64, 64, 1)[0]
        px = 0.2126 * fx[0] + 0.7152 * fx[1] + 0.0722 * fx[2]
        py = 0.2126 * fy[0] + 0.7152 * fy[1] + 0.0722 * fy[2]
        lhs = px * _kelemen_density(delta, sx, s1, s2) * ch.accept_prob(x, y, px, py)
        rhs = py * _kelemen_density(-delta, sy, s1, s2) * ch.accept_prob(y, x, py, px)
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=0.0)
        checked += 1
        across += kx != ky
    assert checked > 3000 and across > 200


def test_chain_invariants(oracle_mod):
    ch = _chains(oracle_mod, 2)
    ch.init()
    ch.run_epochs(20)
    assert len(ch.hist) == 16
    assert int(ch.hist.sum()) == 32 * 8 * 20
    assert (ch.hist > 0).sum() > 8
