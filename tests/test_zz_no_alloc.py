"""pp_voxelize_static (no device allocation, scratch in a static device array) against
pp_voxelize (caller workspace), through the C ABI.

Some callers cannot allocate device memory once they run -- real-time threads whose
allocation calls could block or synchronise the device, or hosts whose device memory belongs
to another framework -- so the library offers this variant.  Voxelisation is integer and copy
work, so the two entry points must agree bit for bit; the check runs on two calls in a row
because the static scratch keeps the previous call's contents.  Named so that pytest collects
it last."""
import numpy as np
import pytest

from pp_synth import GEOM_FULL, GEOM_SMALL, config_points, uniform_cloud

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
import paper_2509_12207_gb300 as pp  # noqa: E402

DEV = "cuda:0"


def _batch(clouds, cap):
    pts = np.zeros((len(clouds), cap, 4), np.float32)
    for i, c in enumerate(clouds):
        pts[i, : len(c)] = c
    return (torch.from_numpy(pts).to(DEV),
            torch.tensor([len(c) for c in clouds], dtype=torch.int32, device=DEV))


def _same(a, b):
    assert torch.equal(a["num_pillars"], b["num_pillars"])
    assert torch.equal(a["cnt"], b["cnt"])
    assert torch.equal(a["pillar_of_cell"], b["pillar_of_cell"])
    for f in range(a["num_pillars"].shape[0]):
        num = int(a["num_pillars"][f])
        for k in ("coord", "npts", "pts"):          # entries past num_pillars are unspecified
            assert torch.equal(a[k][f, :num], b[k][f, :num])


def test_static_scratch_matches_workspace_variant():
    cases = [
        (GEOM_SMALL, [config_points(3, 0, 150000), config_points(3, 1, 31000), np.zeros((0, 4), np.float32),
                      uniform_cloud(5000, 9, GEOM_SMALL)], 150000),
        (GEOM_FULL, [config_points(2, 0)], 120000),
    ]
    for g, clouds, cap in cases:
        pts, n = _batch(clouds, cap)
        ref = pp.voxelize(pts, n, g)
        for _ in range(2):                           # two calls in a row share the scratch
            got = pp.voxelize_static(pts, n, g)
            torch.cuda.synchronize()
            _same(got, ref)
            for f, c in enumerate(clouds):
                assert torch.equal(got["cell"][f, : len(c)], ref["cell"][f, : len(c)])


def test_static_scratch_rejects_oversized_batch():
    g = GEOM_SMALL
    pts = torch.zeros((16, 150000, 4), dtype=torch.float32, device=DEV)   # needs > 16 MiB
    n = torch.zeros((16,), dtype=torch.int32, device=DEV)
    with pytest.raises(pp.PPError) as e:
        pp.voxelize_static(pts, n, g)
    assert e.value.code == pp.PP_EINVAL and "scratch" in str(e.value)
