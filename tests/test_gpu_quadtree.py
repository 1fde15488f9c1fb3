"""RA-Quadtree partition (Sec. 6.2) on the GPU against the oracle: every
mutation replayed; the tree (children, leaf ids, depths) and the region
tables after every refinement pass must match exactly."""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu

# the most mutations each window may let through, measured on a GB300
PINS = {"toy": {}, "cornell": {"f_bounded": 10}}

QT = dict(partition=1, qt_max_leaves=256, qt_max_depth=6)


def _run(oracle_mod, scene=None, toy=None, n_epochs=40, pin="toy", **params):
    from gpu_run import traced_run, replay_full, check_counters
    gpu = traced_run(scene=scene, toy=toy, n_epochs=n_epochs, **params)
    osc = oracle_mod.Scene(toy=toy) if toy is not None else oracle_mod.Scene(scene, use_bvh=False)
    ch, rp, adopted = replay_full(oracle_mod, gpu, osc)
    check_counters(ch, gpu, rp, PINS[pin], adopted, 0)
    child_g, leaf_g, depth_g = gpu["quadtree"]
    child_o, leaf_o, depth_o = ch.quadtree()
    assert np.array_equal(child_g, child_o) and np.array_equal(leaf_g, leaf_o)
    assert np.array_equal(depth_g, depth_o)
    return gpu, ch


def test_quadtree_toy_full_trajectory(oracle_mod):
    gpu, ch = _run(oracle_mod, toy=S.TOY_DEFAULT, n_epochs=60, n_chains=128, width=64, height=64,
                   region_px=8, max_depth=0, epoch_len=16, n_bootstrap=1 << 12, p_large=0.2,
                   qt_split=600, qt_refine=128 * 16 * 4, **QT)
    assert gpu["stats"]["n_regions"] > 20


def test_quadtree_cornell_full_trajectory(oracle_mod):
    gpu, ch = _run(oracle_mod, scene=S.cornell_box(), n_epochs=80, n_chains=64, epoch_len=16, pin="cornell",
                   n_bootstrap=1 << 14, qt_split=400, qt_refine=64 * 16 * 5, **QT)
    assert gpu["stats"]["n_regions"] > 10


def test_quadtree_rejects_weighted_target():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.cornell_box())
    with pytest.raises(rmlt.RmltError):
        R.init_chains(target_mode=1, **QT)


def test_quadtree_checkpoint_resume(tmp_path):
    from paper_2402_08273_gb300 import rmlt
    params = dict(n_chains=256, width=64, height=64, max_depth=4, n_bootstrap=1 << 12, qt_split=300,
                  qt_refine=256 * 16 * 3, **QT)

    def run(steps):
        R = rmlt.Renderer()
        R.load_scene(S.cornell_box())
        R.init_chains(**params)
        for n in steps:
            R.step(n)
        return R

    A = run([160, 160])
    B = run([160])
    B.save(tmp_path / "q.ckpt")
    B.close()
    C = run([])
    C.restore(tmp_path / "q.ckpt")
    C.step(160)
    for a, c in zip(A.read_quadtree(), C.read_quadtree()):
        assert np.array_equal(a, c)
    assert np.array_equal(A.read_region_hist(), C.read_region_hist())
    assert np.array_equal(A.read_chain_state()["q"], C.read_chain_state()["q"])
    assert np.array_equal(A.read_region_params()["lambda"], C.read_region_params()["lambda"])
