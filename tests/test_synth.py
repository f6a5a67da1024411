"""The seeded input generator: determinism, random access, distributions."""
import numpy as np

from paper_2408_03452_gb300 import synth


def test_splitmix_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (state += GAMMA, then the finaliser) are 0xE220A8397B1DCDAF,
    # 0x6E789E6AA1B965F4, 0x06C45D188009454F.
    z = np.array([1, 2, 3], dtype=np.uint64) * synth.GAMMA
    out = synth._mix(z)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_based_random_access():
    full = synth.lognormal_field(9, 7, 20, 1.5, seed=3, layer=8)
    cells = np.array([0, 5, 63, 200, 9 * 7 * 20 - 1])
    np.testing.assert_array_equal(synth.lognormal_at(9, 7, 20, 1.5, 3, cells, layer=8), full[cells])
    full1 = synth.lognormal_field(9, 7, 20, 1.0, seed=3)
    np.testing.assert_array_equal(synth.lognormal_at(9, 7, 20, 1.0, 3, cells), full1[cells])


def test_layer_correlation_structure():
    nx, ny, nz = 6, 5, 19
    K = synth.lognormal_field(nx, ny, nz, 1.5, seed=1, layer=8).reshape(nz, ny, nx)
    for k in range(nz):
        np.testing.assert_array_equal(K[k], K[(k // 8) * 8])
    assert not np.array_equal(K[0], K[8])


def test_distribution_moments():
    n = 200_000
    z = synth.normal(7, synth.STREAM_LNK, np.arange(n))
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    lk = np.log(synth.lognormal_field(100, 100, 20, 1.5, seed=2))
    assert abs(lk.mean()) < 0.02 and abs(lk.std() - 1.5) < 0.02
    u = synth.uniform(1, 2, np.arange(n))
    assert 0.0 < u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


def test_seeds_and_streams_differ():
    a = synth.uniform(0, 1, np.arange(100))
    assert not np.array_equal(a, synth.uniform(1, 1, np.arange(100)))
    assert not np.array_equal(a, synth.uniform(0, 2, np.arange(100)))


def test_boundary_and_wells():
    mask, pD = synth.dirichlet_faces(4, 3, 2, "x", 1.0, 0.0)
    m = mask.reshape(2, 3, 4)
    assert m[:, :, 0].all() and m[:, :, -1].all() and not m[:, :, 1:-1].any()
    idx, val = synth.well_pair(4, 3, 2)
    assert idx.tolist() == [0, 23] and val.tolist() == [1.0, -1.0]


def test_channels_multiply_once():
    nx, ny, nz = 40, 30, 20
    m = synth.channel_mask(nx, ny, nz, 1, n_channels=6, width=4, thickness=6, amplitude=5.0,
                           wavelength=20.0)
    base = synth.lognormal_field(nx, ny, nz, 1.0, 1).reshape(nz, ny, nx)
    K = synth.channelized_field(nx, ny, nz, 1.0, 1, n_channels=6, width=4, thickness=6,
                                amplitude=5.0, wavelength=20.0, contrast=1e3).reshape(nz, ny, nx)
    assert m.any() and not m.all()
    np.testing.assert_allclose(K[m], 1e3 * base[m])
    np.testing.assert_array_equal(K[~m], base[~m])


def test_ensemble_generator_recipe():
    ens = synth.ensemble(seed=1, n_inst=24)
    assert len(ens) == 24
    assert {(w["nx"], w["ny"], w["nz"]) for w in ens} <= set(synth.ENSEMBLE_SIZES)
    assert all(0.5 <= w["sigma"] <= 2.5 and 0.5 <= w["p_hi"] <= 2.0 for w in ens)
    assert len({w["axis"] for w in ens}) > 1
    assert len({(w["nx"], w["ny"], w["nz"]) for w in ens}) > 1
