"""Seeded input generators: the random stream against its published definition,
and each workload's fields against the recipe its docstring states.

These run on the CPU only; the generators hold none of the method's arithmetic.
"""
import numpy as np
import pytest

from paper_2411_09244_gb300 import inputs as I


def test_splitmix64_published_vectors():
    # splitmix64 (Steele, Lea, Flood 2014) in the form of Vigna's public
    # reference code: its first outputs from seed 1234567 and from seed 0.
    r = I.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    assert I.SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF


def test_uniform_and_randint_ranges():
    r = I.SplitMix64(99)
    u = np.array([r.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    # The top 53 bits scaled by 2**-53: every draw is an exact multiple of 2**-53.
    assert np.all(np.floor(u * 2.0 ** 53) == u * 2.0 ** 53)
    k = np.array([r.randint(3, 7) for _ in range(20000)])
    assert k.min() == 3 and k.max() == 7
    counts = np.bincount(k - 3, minlength=5)
    assert np.all(np.abs(counts / len(k) - 0.2) < 0.02)
    assert all(r.randint(4, 4) == 4 for _ in range(10))


@pytest.mark.parametrize("make", [I.config_c1, I.config_c2, I.config_c3, I.config_paper_grid,
                                  lambda: I.config_c4(5), lambda: I.config_small(n_f=24, seed=3)])
def test_configs_are_deterministic_and_well_formed(make):
    a, b = make(), make()
    for name in ("kappa", "f", "u0", "amp"):
        assert np.array_equal(getattr(a, name), getattr(b, name))
    n_f = a.n_f
    nn = (n_f + 1) ** 2
    assert a.kappa.shape == (n_f, n_f)
    assert a.f.shape == (nn,) and a.u0.shape == (nn,)
    assert a.amp.shape == (a.N,)
    assert n_f % a.nc == 0
    assert np.all(np.isfinite(a.kappa)) and a.kappa.min() == 1.0
    # u0 vanishes on the Dirichlet boundary.
    g = a.u0.reshape(n_f + 1, n_f + 1)
    assert not g[0].any() and not g[-1].any() and not g[:, 0].any() and not g[:, -1].any()


def test_instances_differ():
    assert not np.array_equal(I.config_c2(0).kappa, I.config_c2(1).kappa)
    assert not np.array_equal(I.config_c3(0).u0, I.config_c3(1).u0)


def test_paint_kappa_values_margin_and_no_gaps():
    n_f = 128
    k = I.paint_kappa(I.SplitMix64(5), n_f, 30, 1e5, 2, n_incl=20, incl_value=1e3)
    assert set(np.unique(k)) <= {1.0, 1e3, 1e5}
    assert (k == 1e5).any() and (k == 1e3).any()
    m = max(1, n_f // 32)
    # Every feature keeps m cells away from the boundary.
    assert np.all(k[:m] == 1) and np.all(k[-m:] == 1)
    assert np.all(k[:, :m] == 1) and np.all(k[:, -m:] == 1)
    # No background cell is left between two high cells in a row or a column.
    hi = k > 1
    lr = hi[:, :-2] & hi[:, 2:] & ~hi[:, 1:-1]
    ud = hi[:-2, :] & hi[2:, :] & ~hi[1:-1, :]
    assert not lr.any() and not ud.any()


def test_close_gaps_fills_one_cell_strips_with_the_larger_neighbour():
    k = np.ones((6, 7))
    k[1, 0] = 10.0
    k[1, 2] = 100.0          # (1, 1) lies between them in a row
    k[3, 5] = 5.0
    k[5, 5] = 7.0            # (4, 5) lies between them in a column
    out = I.close_gaps(k)
    expect = k.copy()
    expect[1, 1] = 100.0
    expect[4, 5] = 7.0
    assert np.array_equal(out, expect)
    assert k[1, 1] == 1.0    # the input is not modified
    # A fill can open a further gap: (1, 1) fills first, then (2, 1) lies
    # between it and (3, 1), and the fill repeats until none is left.
    k2 = np.ones((4, 3))
    k2[1, 0] = k2[1, 2] = 5.0
    k2[3, 1] = 8.0
    expect2 = k2.copy()
    expect2[1, 1] = 5.0
    expect2[2, 1] = 8.0
    assert np.array_equal(I.close_gaps(k2), expect2)


def test_c3_source_and_amplitudes():
    p = I.config_c3()
    assert p.N == 32 and p.P == 32
    a16 = p.meta["amp16"]
    assert a16.shape == (16,) and a16.min() >= 0.5 and a16.max() < 1.5
    # Each of the 16 amplitudes is held over two consecutive intervals.
    assert np.array_equal(p.amp[0::2], a16) and np.array_equal(p.amp[1::2], a16)
    # One Gaussian at the centre: its maximum is 1 at the centre node.
    c = (p.n_f // 2) * (p.n_f + 1) + p.n_f // 2
    assert p.f[c] == 1.0 and p.f.max() == 1.0


def test_c4_instance_draws_stay_in_documented_ranges():
    for i in range(12):
        p = I.config_c4(i)
        assert p.n_f in (64, 96, 128, 192, 256)
        assert p.nc == p.n_f // 8 and p.P == 32 and p.ell == 2
        assert 2 <= p.J <= 4 and p.N in (16, 32, 64)
        assert 1e3 <= p.meta["contrast"] < 1e6
        assert 5 <= p.meta["channels"] <= 50 and 5 <= p.meta["inclusions"] <= 50
        assert p.eps < 0   # relative jump tolerance
        assert not p.u0.any()


def test_observation_nodes_distinct_interior():
    n_f = 64
    nodes = I.observation_nodes(n_f, 40, seed=2)
    assert len(np.unique(nodes)) == 40
    i, j = nodes % (n_f + 1), nodes // (n_f + 1)
    assert i.min() >= 1 and i.max() <= n_f - 1 and j.min() >= 1 and j.max() <= n_f - 1
    assert np.array_equal(nodes, I.observation_nodes(n_f, 40, seed=2))
