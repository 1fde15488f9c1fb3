"""The oracle's starting states (CPU, no GPU).

Each chain takes the bootstrap sample where the cumulative sum of pi over all
n_bootstrap uniform samples first exceeds its point (g + u_g) / C of the total
(systematic resampling in proportion to pi).  Pinned here:
  - a chain never starts on a path that contributes nothing while some sample
    contributes, even with one bootstrap sample per chain (a chain that
    resampled only its own slice of samples started on a black path whenever
    the slice held no contributing one, and its mutations then added nothing
    to the image until it left it);
  - the starting states follow pi: on the toy integrand their histogram over
    the screen regions matches the closed-form region masses;
  - the choice is the cumulative-sum crossing, recomputed here from the
    bootstrap samples' own contributions.
"""
import numpy as np

from paper_2402_08273_gb300 import scenes as S

TOY = S.TOY_DEFAULT


def _tv(p, q):
    return 0.5 * float(np.abs(p - q).sum())


def _boot_words(oracle_mod, s, D, seed):
    """Bootstrap sample s: its D words, drawn from the counter {s, 0, ~0, 0x8000 + j}."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w = np.concatenate([oracle_mod.philox4x32_10([s & 0xFFFFFFFF, s >> 32, 0xFFFFFFFF, 0x8000 + j], key)
                        for j in range((D + 3) // 4)])
    return w[:D]


def _lum(f):
    return 0.2126 * f[0] + 0.7152 * f[1] + 0.0722 * f[2]


def test_every_chain_starts_on_a_contributing_path(oracle_mod):
    # direct light only: the ceiling and the shadowed floor contribute nothing
    sc = oracle_mod.Scene(S.cornell_box(), use_bvh=False)
    ch = oracle_mod.Chains(sc, n_chains=256, width=32, height=32, region_px=8, max_depth=1, epoch_len=4,
                           n_bootstrap=256, p_large=0.3, seed=3)
    ch.init()
    pis = np.array([_lum(sc.path_eval(_boot_words(oracle_mod, s, ch.D, 3), 32, 32, 1)[0]) for s in range(256)])
    assert (pis == 0).sum() > 10 and (pis > 0).sum() > 10
    assert (ch.pi > 0).all()
    # the chosen samples are the crossings of the cumulative sum
    cum = np.cumsum(pis)
    for g in range(256):
        s = int(ch.boot_choice[g])
        u = (int(oracle_mod.philox4x32_10([g, 0, 0xFFFFFFFF, 0x7FFE], [3, 0])[0]) >> 8) * 2.0 ** -24
        t = (g + u) / 256 * cum[-1]
        assert cum[s] > t and (s == 0 or cum[s - 1] <= t)


def test_starting_states_follow_pi_on_the_toy(oracle_mod):
    sc = oracle_mod.Scene(toy=TOY)
    ch = oracle_mod.Chains(sc, n_chains=1 << 16, width=64, height=64, region_px=8, max_depth=0, epoch_len=4,
                           n_bootstrap=1 << 18, p_large=0.3, seed=11)
    ch.init()
    h = np.bincount(ch.k, minlength=64).astype(float)
    b = S.toy_region_masses(TOY, 64, 64, 8)
    # 2^16 chains over 64 regions of masses 0.3 % to 93 %: sampling noise
    # alone gives a total variation near 0.01 (0.018 at 2^14 chains, whatever
    # the bootstrap size); uniform starting states would give about 0.7
    assert _tv(h / h.sum(), b / b.sum()) < 0.02
