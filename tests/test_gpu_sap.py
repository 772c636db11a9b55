"""GPU parity for adaptive patching and the 2-bit masks (Sec. V-B(c),
Eq. (1); Sec. V-C(a)) against the SAP oracle, bit for bit: every decision
is integer or a fixed sequence of IEEE operations on both sides."""
import numpy as np
import pytest

from oracle import sap
from gpu_util import fbp_api, needs_gpu, torch
from paper_2505_13955_gb300 import phantoms

pytestmark = [pytest.mark.gpu, needs_gpu]


def to_dev16(img):
    return torch.from_numpy(np.ascontiguousarray(img, dtype=np.uint16).view(np.int16)).cuda()


def random_slice(n, seed):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 3000, (n, n)).astype(np.uint16)
    yy, xx = np.mgrid[0:n, 0:n]
    for _ in range(8):
        cx, cy, rad = rng.uniform(0, n, 2).tolist() + [rng.uniform(n / 10, n / 3)]
        img[(xx - cx) ** 2 + (yy - cy) ** 2 < rad ** 2] += np.uint16(rng.integers(5000, 20000))
    return img


def thresholds(img):
    gx, gy = sap.sobel(sap.smooth(img))
    m = np.abs(gx) + np.abs(gy)
    return int(np.percentile(m, 80)), int(np.percentile(m, 95))


@pytest.mark.parametrize("n,seed", [(16, 1), (64, 2), (128, 3), (256, 4)])
def test_edges_match_oracle(n, seed):
    api = fbp_api()
    img = random_slice(n, seed)
    lo, hi = thresholds(img)
    p = api.SapParams(n, patch=4, length=1, canny_lo=lo, canny_hi=hi)
    e = api.sap_edges(to_dev16(img), p).cpu().numpy()
    ref = sap.canny(img, lo, hi)
    np.testing.assert_array_equal(e, ref)
    assert 0 < ref.sum() < n * n
    assert api.device_status() == 0


def test_edges_of_a_phantom_slice_and_threshold_extremes():
    api = fbp_api()
    img = phantoms.sap_slice(512, 31)
    c = phantoms.SAP
    for lo, hi in [(c["canny_lo"], c["canny_hi"]), (0, 0), (0, 2 ** 31 - 1), (2 ** 31 - 1, 2 ** 31 - 1)]:
        p = api.SapParams(512, 16, 1, lo, hi)
        np.testing.assert_array_equal(api.sap_edges(to_dev16(img), p).cpu().numpy(), sap.canny(img, lo, hi))


@pytest.mark.parametrize("n,P,length,seed", [(16, 4, 1, 5), (16, 4, 16, 6), (64, 4, 100, 7), (64, 8, 64, 8),
                                             (256, 16, 88, 9), (256, 4, 2209, 10), (512, 16, 511, 11),
                                             (512, 64, 64, 12)])
def test_patches_match_oracle(n, P, length, seed):
    api = fbp_api()
    img = random_slice(n, seed)
    lo, hi = thresholds(img)
    p = api.SapParams(n, P, length, lo, hi)
    d = to_dev16(img)
    e = api.sap_edges(d, p)
    patches, leaves = api.sap_patches(d, e, p)
    ref_e = sap.canny(img, lo, hi)
    ref_leaves, _ = sap.quadtree(img, ref_e, P, length)
    np.testing.assert_array_equal(leaves.cpu().numpy(), np.array(ref_leaves, dtype=np.int32).reshape(-1, 3))
    np.testing.assert_array_equal(patches.cpu().numpy(), sap.extract_patches(img, ref_leaves, P))
    assert api.device_status() == 0


def test_host_stack_overlapped_streams_match_oracle():
    """sap_host: a stack of pinned host slices through two streams gives,
    slice by slice, the oracle's leaves and patches (odd count: one stream
    takes an extra slice)."""
    api = fbp_api()
    n, P, length, S = 128, 8, 97, 5
    imgs = np.stack([random_slice(n, 40 + i) for i in range(S)])
    lo, hi = thresholds(imgs[0])
    p = api.SapParams(n, P, length, lo, hi)
    host = torch.from_numpy(imgs.view(np.int16)).pin_memory()
    patches, leaves = api.sap_host(host, p)
    assert not patches.is_cuda and not leaves.is_cuda
    for i in range(S):
        ref_leaves, _ = sap.quadtree(imgs[i], sap.canny(imgs[i], lo, hi), P, length)
        np.testing.assert_array_equal(leaves[i].numpy(), np.array(ref_leaves, dtype=np.int32).reshape(-1, 3))
        np.testing.assert_array_equal(patches[i].numpy(), sap.extract_patches(imgs[i], ref_leaves, P))
    assert api.device_status() == 0


def test_constant_slice_splits_by_morton_order():
    """No edges and no variance: every key ties, so the order is level, then
    Morton code -- the tree is the first splits of a breadth-first Z-order."""
    api = fbp_api()
    img = np.full((64, 64), 1234, dtype=np.uint16)
    p = api.SapParams(64, 4, 40, 1, 2)
    d = to_dev16(img)
    patches, leaves = api.sap_patches(d, api.sap_edges(d, p), p)
    ref, _ = sap.quadtree(img, np.zeros((64, 64), np.uint8), 4, 40)
    np.testing.assert_array_equal(leaves.cpu().numpy(), np.array(ref, dtype=np.int32).reshape(-1, 3))
    assert np.all(patches.cpu().numpy() == 1234.0)


@pytest.mark.parametrize("n,P,length", [(64, 4, 100), (256, 16, 121), (128, 8, 256)])
def test_depatch_pack_matches_oracle(n, P, length):
    api = fbp_api()
    img = random_slice(n, n + P)
    lo, hi = thresholds(img)
    p = api.SapParams(n, P, length, lo, hi)
    d = to_dev16(img)
    _, leaves = api.sap_patches(d, api.sap_edges(d, p), p)
    rng = np.random.default_rng(n)
    mp = rng.integers(0, 256, (length, P, P)).astype(np.uint8)      # high bits are ignored
    packed = api.sap_depatch_pack(torch.from_numpy(mp).cuda(), leaves, p).cpu().numpy()
    lv = [tuple(x) for x in leaves.cpu().numpy().tolist()]
    ref = sap.pack2(sap.depatch(mp & 3, lv, n, P))
    np.testing.assert_array_equal(packed, ref)
    assert api.device_status() == 0


def test_depatch_rejects_leaves_outside_the_slice():
    """A leaf entry outside the slice is skipped and reported through the
    device status word; the other leaves are still written."""
    api = fbp_api()
    n, P = 64, 16
    p = api.SapParams(n, P, 16, 1, 2)
    good = [(x, y, 16) for y in range(0, 64, 16) for x in range(0, 64, 16)]
    lv = np.array(good, dtype=np.int32)
    lv[5] = (64, 0, 16)                    # starts past the right edge
    lv[9] = (8, 16, 16)                    # not aligned to its side
    mp = np.full((16, P, P), 2, dtype=np.uint8)
    out = torch.zeros((n, n // 4), dtype=torch.uint8, device="cuda")
    api.sap_depatch_pack(torch.from_numpy(mp).cuda(), torch.from_numpy(lv).cuda(), p, out=out)
    assert api.device_status() == 5
    got = sap.unpack2(out.cpu().numpy())
    for i, (x0, y0, s) in enumerate(good):
        expect = 0 if i in (5, 9) else 2
        assert np.all(got[y0:y0 + s, x0:x0 + s] == expect)
    assert api.device_status() == 0


def test_sap_full_size_slice():
    """The benchmark's configuration (n = 8192, P = 16, 4096 patches) on one
    phantom slice: edges, leaves and patches bit-exact."""
    api = fbp_api()
    c = phantoms.SAP
    img = phantoms.sap_slice(8192, phantoms.slice_seed(9, 0))
    p = api.SapParams(8192, c["patch"], c["length"], c["canny_lo"], c["canny_hi"])
    d = to_dev16(img)
    e = api.sap_edges(d, p)
    patches, leaves = api.sap_patches(d, e, p)
    ref_e = sap.canny(img, c["canny_lo"], c["canny_hi"])
    np.testing.assert_array_equal(e.cpu().numpy(), ref_e)
    ref_leaves, _ = sap.quadtree(img, ref_e, c["patch"], c["length"])
    np.testing.assert_array_equal(leaves.cpu().numpy(), np.array(ref_leaves, dtype=np.int32).reshape(-1, 3))
    np.testing.assert_array_equal(patches.cpu().numpy(), sap.extract_patches(img, ref_leaves, c["patch"]))
    assert api.device_status() == 0
