"""Image preparation on the GPU vs the numpy oracle, bit for bit:
mixing region (Sec. 4.2) and mixed-wet relabel (Sec. 3.3)."""
import numpy as np
import pytest

from oracle import prepare

pytestmark = pytest.mark.gpu


def _image(shape, seed, solid=0.6):
    rng = np.random.default_rng(seed)
    lab = np.where(rng.uniform(size=shape) < solid, rng.integers(1, 4, size=shape), 0).astype(np.uint16)
    return lab, rng


@pytest.mark.parametrize("shape,axis,n_mix", [((9, 7, 13), 2, 3), ((9, 7, 13), 0, 6), ((9, 7, 13), 1, 1),
                                               ((40, 33, 65), 2, 8), ((1, 1, 2), 0, 1)])
def test_mixing_layer_matches_oracle(shape, axis, n_mix):
    import paper_2007_12266_gb300 as lbm
    lab, _ = _image(shape, 11 + n_mix)
    want = prepare.mixing_layer(lab, axis, n_mix)
    got = lbm.mixing_layer(lab, n_mix, axis=axis)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1), (1, 0, 1), (0, 1, 0)])
@pytest.mark.parametrize("radius", [1.0, 2.0, 2.5, 3.7])
def test_mixed_wet_relabel_matches_oracle(periodic, radius):
    import paper_2007_12266_gb300 as lbm
    lab, rng = _image((11, 14, 19), 23)
    oil = (rng.uniform(size=lab.shape) < 0.04) & (lab == 0)
    want = prepare.mixed_wet_relabel(lab, oil, periodic, radius, 7)
    got = lbm.mixed_wet_relabel(lab, oil, radius=radius, new_label=7, periodic=periodic)
    assert np.array_equal(got, want)


def test_mixed_wet_relabel_full_size_sample():
    """A 128^3 sphere pack with a blob oil phase: whole-image equality."""
    import paper_2007_12266_gb300 as lbm
    from synthetic import phi0_blob, sphere_pack
    lab = sphere_pack(128, 0.3, 6.0, 1.5, 77).labels
    phi = phi0_blob(lab, 0.5, 78)
    oil = (phi < 0) & (lab == 0)
    want = prepare.mixed_wet_relabel(lab, oil, (1, 1, 1), 2.0, 2)
    got = lbm.mixed_wet_relabel(lab, oil, radius=2.0, new_label=2, periodic=(1, 1, 1))
    assert np.array_equal(got, want)
    assert np.count_nonzero(got == 2) > 0


def test_invalid_arguments_are_rejected():
    import paper_2007_12266_gb300 as lbm
    lab, _ = _image((6, 6, 6), 1)
    with pytest.raises(lbm.LBPMError):
        lbm.mixing_layer(lab, 4, axis=2)          # 2 * n_mix > extent
    with pytest.raises(lbm.LBPMError):
        lbm.mixing_layer(lab, 1, axis=3)
    with pytest.raises(lbm.LBPMError):
        lbm.mixed_wet_relabel(lab, lab == 0, radius=9.0)
    with pytest.raises(lbm.LBPMError):
        lbm.mixed_wet_relabel(lab, lab == 0, new_label=0)
