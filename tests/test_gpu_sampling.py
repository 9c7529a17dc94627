"""GPU parity of hierarchical NDF importance sampling (row f1, Sec. 5.2)
against the FP64 oracle on the same uniforms, and the check of Fig.
sampleNDF: the histogram of 10^7 GPU samples is the normalised NDF image."""
import numpy as np
import pytest
import torch

import synth
from oracle import sampling as osm
from _gpu import dev, lib, oracle_material, random_factors

pytestmark = pytest.mark.gpu

# (N, rank, bins): the batching materials with power-of-two bins <= 64
SHAPES = [(128, 16, 16), (128, 32, 64), (256, 16, 32), (256, 64, 32), (512, 32, 16), (1024, 64, 32)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _materials(signed, shapes=SHAPES, seed=500):
    import paper_2109_14807_gb300 as g
    mats, omats, dims = [], [], []
    for i, (N, R, B) in enumerate(shapes):
        L = int(np.log2(N)) + 1
        f = random_factors(N, L, B, R, seed + i, signed=signed)
        mat = g.QueryMaterial.from_factors({k: dev(v) for k, v in f.items()})
        g.build_query_tables(mat)
        mats.append(mat)
        omats.append(oracle_material(f))
        dims.append((N, L, B))
    return mats, omats, dims


def _footprints(dims, per, seed):
    parts = []
    for m, (N, L, B) in enumerate(dims):
        parts.append(synth.sample_footprints(N, L, per, seed + m, material=m))
    return np.concatenate(parts)


def test_sampling_matches_oracle_on_the_same_uniforms():
    import paper_2109_14807_gb300 as g
    mats, omats, dims = _materials(signed=True)
    s = _footprints(dims, 2500, 40)
    n = len(s)
    u = synth.sample_uniforms(31, n)
    st = g.new_status()
    got = g.sample_ndf(mats, g.samples_to_device(s), dev(u), status=st).cpu().numpy().astype(np.float64)
    assert g.status_bits(st) == 0
    ref = osm.sample_batch(omats, s, u.astype(np.float64))
    gb = np.floor(got[:, :2]).astype(np.int64)
    rb = np.floor(ref[:, :2]).astype(np.int64)
    same = np.all(gb == rb, axis=1)
    # FP32 sums can flip a choice only where the oracle's u * total lay within
    # rounding of a cumulative boundary
    assert np.all(same | (ref[:, 4] < 1e-4)), np.nonzero(~same & (ref[:, 4] >= 1e-4))[0][:5]
    assert same.mean() > 0.995
    m = same
    assert np.max(np.abs(got[m, 2] - ref[m, 2])) <= 1e-4
    # the bin value: error relative to the magnitude of the rank terms
    kap = np.array([np.sum(np.abs(osm.footprint_weights(omats[int(s[i]["material"])], int(s[i]["x"]),
                                                        int(s[i]["y"]), float(s[i]["level"]))
                                  * omats[int(s[i]["material"])]["fs"][rb[i, 0]]
                                  * omats[int(s[i]["material"])]["ft"][rb[i, 1]]))
                    for i in np.nonzero(m)[0]])
    err = np.abs(got[m, 3] - ref[m, 3]) / np.maximum(kap, 1e-30)
    assert np.max(err) <= 1e-5
    assert np.all((got[:, 0] < np.array([d[2] for d in dims])[s["material"]]) & (got[:, 0] >= 0))
    # the sample sits at bin + (u6, u7)
    assert np.max(np.abs(got[:, 0] - (gb[:, 0] + u[:, 6]))) <= 1e-4
    assert np.max(np.abs(got[:, 1] - (gb[:, 1] + u[:, 7]))) <= 1e-4


def test_histogram_of_ten_million_samples_is_the_ndf_image():
    # Fig. sampleNDF: sampling by range queries reproduces the NDF image
    import paper_2109_14807_gb300 as g
    mats, omats, dims = _materials(signed=False, shapes=[(256, 16, 16)], seed=800)
    n = 10_000_000
    x, y, level = 37, 101, 3.4
    s = np.zeros(n, dtype=synth.SAMPLE_DTYPE)
    s["x"], s["y"], s["level"] = x, y, level
    u = synth.sample_uniforms(77, n)
    out = g.sample_ndf(mats, g.samples_to_device(s), dev(u))
    B = dims[0][2]
    bins = out[:, 0].floor().long() * B + out[:, 1].floor().long()
    cnt = torch.bincount(bins, minlength=B * B).double().cpu().numpy().reshape(B, B)
    pmf = osm.bin_pmf(omats[0], x, y, level)
    img = osm.ndf_image(omats[0], x, y, level)
    assert np.allclose(pmf, img / img.sum(), rtol=1e-12)  # non-negative material
    exp = n * pmf
    chi2 = float(((cnt - exp) ** 2 / exp).sum())
    dof = B * B - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), chi2
    # the pmf each sample reports is its bin's probability
    got_pmf = out[:, 2].double().cpu().numpy()
    b = bins.cpu().numpy()
    assert np.max(np.abs(got_pmf - pmf.ravel()[b]) / pmf.ravel()[b]) <= 1e-5


def test_malformed_and_unsupported():
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300._lib import GspError
    mats, omats, dims = _materials(signed=True, shapes=[(64, 16, 16)], seed=900)
    s = np.zeros(3, dtype=synth.SAMPLE_DTYPE)
    s["material"] = [0, 5, 0]
    s["level"] = [1.0, 1.0, np.nan]
    u = synth.sample_uniforms(3, 3)
    st = g.new_status()
    out = g.sample_ndf(mats, g.samples_to_device(s), dev(u), status=st).cpu().numpy()
    assert np.all(np.isfinite(out[0])) and np.all(np.isnan(out[1])) and np.all(np.isnan(out[2]))
    assert g.status_bits(st) & 0x2
    empty = g.sample_ndf(mats, g.samples_to_device(s[:0]), dev(u[:0]))
    assert empty.shape == (0, 4)
    odd, _, _ = _materials(signed=True, shapes=[(64, 16, 24)], seed=901)  # 24 bins: not a power of two
    with pytest.raises(GspError):
        g.sample_ndf(odd, g.samples_to_device(s[:1]), dev(u[:1]))
