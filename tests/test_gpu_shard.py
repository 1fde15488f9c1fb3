"""Sharded populations on one GPU: contexts that split the chains by global
id and sum their region statistics between epochs (rmlt_epoch_mutate /
rmlt_epoch_update around an addition of the exchange buffers, which is what
an all-reduce over GPUs computes) equal one context stepping the whole
population with rmlt_step.  Integer tables, lambda, weights, the quadtree and
every chain's state are compared bit for bit; the image shares sum to the
image within the binary64 splat tolerance."""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu

CASES = {
    "cornell": dict(scene=lambda: S.cornell_box(), epochs=8,
                    params=dict(n_chains=256, width=64, height=64, region_px=8, max_depth=5,
                                n_bootstrap=1 << 12, seed=3)),
    "two_rooms_bvh": dict(scene=lambda: S.two_rooms(20_000, seed=4), epochs=6,
                          params=dict(n_chains=2048, width=128, height=128, region_px=16, max_depth=8,
                                      n_bootstrap=1 << 13, seed=5)),
    "toy_weighted": dict(toy=S.TOY_DEFAULT, epochs=20,
                         params=dict(n_chains=512, width=32, height=32, region_px=8, max_depth=0,
                                     n_bootstrap=1 << 12, seed=6, target_mode=1)),
    "toy_quadtree": dict(toy=S.TOY_DEFAULT, epochs=20,
                         params=dict(n_chains=512, width=32, height=32, region_px=8, max_depth=0,
                                     n_bootstrap=1 << 12, seed=7, partition=1, qt_max_leaves=256,
                                     qt_max_depth=6, qt_split=300, qt_refine=20_000)),
}


def _renderer(case, wavefront=False, **kw):
    from paper_2402_08273_gb300 import rmlt
    c = CASES[case]
    R = rmlt.Renderer()
    if "toy" in c:
        R.load_toy_integrand(c["toy"])
    else:
        R.load_scene(c["scene"]())
    if wavefront:
        R.set_tuning(wavefront=True)
    R.init_chains(**dict(c["params"], **kw))
    return R


def _tables(R):
    reg = R.read_region_params()
    out = dict(h=R.read_region_hist(), i=reg["i"], A=reg["A"], n=reg["n"], lam=reg["lambda"], w=reg["w"],
               st=R.read_chain_state(), img=R.read_image())
    if R.params["partition"] == 1:
        out["tree"] = R.read_quadtree()
    return out


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("n_shards", [2, 3])
def test_shards_equal_one_context(case, n_shards):
    import torch
    c = CASES[case]
    C = c["params"]["n_chains"]
    one = _renderer(case)
    one.step(c["epochs"] * one.params["epoch_len"])
    ref = _tables(one)
    one.close()
    # uneven shards: the first ones one chain longer
    sizes = [C // n_shards + (1 if r < C % n_shards else 0) for r in range(n_shards)]
    firsts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
    Rs = [_renderer(case, wavefront=(r == 1 and "toy" not in c), n_chains=int(sizes[r]),
                    chain_first=int(firsts[r]), chains_total=C) for r in range(n_shards)]
    bufs = [R.exchange_buffers() for R in Rs]
    for _ in range(c["epochs"]):
        for R, (cn, sm) in zip(Rs, bufs):
            R.epoch_mutate(cn, sm)
        torch.cuda.synchronize()
        tot_c = sum(b[0] for b in bufs)          # int64 addition wraps like u64
        tot_s = sum(b[1] for b in bufs)
        for R in Rs:
            R.epoch_update(tot_c, tot_s)
    torch.cuda.synchronize()
    got = [_tables(R) for R in Rs]
    for r, g in enumerate(got):
        for key in ("h", "i", "A", "n", "lam", "w"):
            assert np.array_equal(g[key], ref[key]), (case, r, key)
        sl = slice(int(firsts[r]), int(firsts[r] + sizes[r]))
        assert np.array_equal(g["st"]["q"], ref["st"]["q"][:, sl]), (case, r, "states")
        assert np.array_equal(g["st"]["k"], ref["st"]["k"][sl]), (case, r, "regions")
        if "tree" in ref:
            for a, b in zip(g["tree"], ref["tree"]):
                assert np.array_equal(a, b), (case, r, "quadtree")
    img = sum(g["img"] for g in got)
    np.testing.assert_allclose(img, ref["img"], rtol=1e-9, atol=1e-9 * max(1.0, float(ref["img"].max())))
    for R in Rs:
        R.close()


def test_unsharded_epoch_calls_equal_step():
    """rmlt_epoch_mutate + rmlt_epoch_update with the buffers passed through
    unchanged is exactly rmlt_step(epoch_len)."""
    a = _renderer("cornell")
    b = _renderer("cornell")
    cn, sm = b.exchange_buffers()
    for _ in range(5):
        a.step(a.params["epoch_len"])
        b.epoch_mutate(cn, sm)
        b.epoch_update(cn, sm)
    ta, tb = _tables(a), _tables(b)
    for key in ("h", "i", "A", "n", "lam"):
        assert np.array_equal(ta[key], tb[key]), key
    assert np.array_equal(ta["st"]["q"], tb["st"]["q"])
    # binary64 splat atomics add in any order
    np.testing.assert_allclose(ta["img"], tb["img"], rtol=1e-12, atol=1e-300)


def test_sharded_context_call_order():
    from paper_2402_08273_gb300 import rmlt
    R = _renderer("cornell", n_chains=128, chain_first=128, chains_total=256)
    with pytest.raises(rmlt.RmltError) as e:
        R.step(16)                       # a shard needs the exchange
    assert e.value.status == -5
    cn, sm = R.exchange_buffers()
    with pytest.raises(rmlt.RmltError) as e:
        R.epoch_update(cn, sm)           # mutate first
    assert e.value.status == -5
    R.epoch_mutate(cn, sm)
    with pytest.raises(rmlt.RmltError) as e:
        R.epoch_mutate(cn, sm)           # update is due
    assert e.value.status == -5
    with pytest.raises(rmlt.RmltError) as e:
        R.epoch_update(cn.cpu(), sm)     # host buffers are refused
    assert e.value.status == -1
    R.epoch_update(cn, sm)
    with pytest.raises(rmlt.RmltError) as e:
        _renderer("cornell", n_chains=128, chain_first=200, chains_total=256)
    assert e.value.status == -1
