"""The seeded input generators: SplitMix64 against its published test vector,
distribution sanity of the uniforms/normals, and the workload recipes."""
import numpy as np

from paper_1905_01330_gb300 import synth


def test_splitmix64_reference_vector():
    # first outputs of SplitMix64 seeded with 1234567 (Vigna's reference implementation)
    assert list(map(int, synth.splitmix64(1234567, 5))) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_counter_form_slices_agree():
    full = synth.splitmix64(99, 100)
    assert np.array_equal(full[40:60], synth.splitmix64(99, 20, offset=40))


def test_uniform_and_normal_moments():
    u = synth.uniform(5, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    z = synth.normal(6, 200000, std=2.0)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 2.0) < 0.02


def test_contraction_specs_respect_recipe():
    specs = synth.contraction_specs(256, seed=2)
    for sha, la, shb, lb in specs:
        assert 3 <= len(sha) <= 5 and 3 <= len(shb) <= 5 and 1 <= len(la) <= 3
        assert len(set(la)) == len(la) and len(set(lb)) == len(lb)
        assert all(sha[a] == shb[b] for a, b in zip(la, lb))
        assert all(d in synth.SPEC_DIMS for d in sha + shb)
        m, n, k = synth.spec_sizes((sha, la, shb, lb))
        assert m * k <= synth.SPEC_CAP and n * k <= synth.SPEC_CAP and m * n <= synth.SPEC_CAP


def test_bonds_and_tfim_shapes():
    assert synth.mps_bonds(6, 2, 4) == [1, 2, 4, 4, 4, 2, 1]
    W = synth.tfim_mpo(4)
    assert [w.shape for w in W] == [(1, 3, 2, 2), (3, 3, 2, 2), (3, 3, 2, 2), (3, 1, 2, 2)]


def test_classifier_separate_mps_is_seeded_and_near_identity():
    a = synth.classifier_separate_mps(8, 4, 3, seed=5, eps_std=0.1)
    b = synth.classifier_separate_mps(8, 4, 3, seed=5, eps_std=0.1)
    assert len(a) == 3 and all(len(m) == 8 for m in a)
    for ma, mb in zip(a, b):
        for x, y in zip(ma, mb):
            assert x.dtype == np.float32 and np.array_equal(x, y)
    assert [c.shape for c in a[0]] == [(1, 2, 4)] + [(4, 2, 4)] * 6 + [(4, 2, 1)]
    assert not np.array_equal(a[0][3], a[1][3])                 # each label its own MPS
    eye = synth.classifier_separate_mps(8, 4, 2, seed=5, eps_std=0.0)[1][3]
    assert np.array_equal(eye[:, 0, :], np.eye(4, dtype=np.float32))
