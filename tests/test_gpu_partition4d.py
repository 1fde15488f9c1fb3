"""The 4-D partition (screen region x a grid over the first bounce's BSDF
coordinates) on the GPU: every mutation of a Cornell-box run replayed by the
oracle with exact region counts, lambda and final states; the wavefront form
reproduces the chain kernel bit for bit."""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu

# the most mutations each window may let through, measured on a GB300
PINS = {"f_bounded": 16}


def test_partition4d_full_trajectory(oracle_mod):
    from gpu_run import traced_run, replay_full, check_counters
    gpu = traced_run(scene=S.cornell_box(), n_epochs=80, n_chains=64, width=64, height=64, region_px=16,
                     max_depth=5, epoch_len=16, n_bootstrap=1 << 14, seed=3, p_large=0.3, dir_cells=3)
    assert gpu["stats"]["n_regions"] == 16 * 9
    ch, rp, adopted = replay_full(oracle_mod, gpu, oracle_mod.Scene(S.cornell_box(), use_bvh=False))
    check_counters(ch, gpu, rp, PINS, adopted, PINS.get("adopted", 0))
    assert rp.s["mutations"] == 64 * 80 * 16
    lam = gpu["region"]["lambda"]
    assert np.count_nonzero(lam != 0.0) > 20        # many 4-D regions adapted


def test_partition4d_wavefront_identical():
    from gpu_run import traced_run
    kw = dict(scene=S.two_rooms(8000, seed=6), n_epochs=3, n_chains=1500, width=96, height=64, region_px=16,
              max_depth=6, epoch_len=16, n_bootstrap=1 << 14, p_large=0.3, dir_cells=2)
    a = traced_run(**kw)
    b = traced_run(tuning={"wavefront": True}, **kw)
    for name in ("f", "a", "qhash", "flags"):
        assert np.array_equal(a["trace"][name], b["trace"][name]), name
    assert np.array_equal(a["final"]["q"], b["final"]["q"])
    assert np.array_equal(a["hist"], b["hist"])


def test_partition4d_parameter_checks():
    from paper_2402_08273_gb300 import rmlt
    R = rmlt.Renderer()
    R.load_scene(S.cornell_box())
    for bad in (dict(dir_cells=2, target_mode=1), dict(dir_cells=2, partition=1), dict(dir_cells=65)):
        with pytest.raises(rmlt.RmltError):
            R.init_chains(n_chains=64, max_depth=3, **bad)
