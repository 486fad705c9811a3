"""hsc_pca_one_band_noalloc: the one-band PCA for callers that cannot
allocate GPU memory while running. Checked through the C ABI against
hsc_pca_one_band on the same cube, on two calls in a row (the second call
reuses the fixed scratch the first one left behind), within the PCA
tolerances of the other GPU tests. Collected last on purpose."""

import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

V1_ANGLE = 1e-5
I_TOL = 2e-5


def test_noalloc_pca_matches_the_context_entry_point(hsc, ctx):
    import torch
    L = hsc.lib()
    f = synth.make_config(2)  # 416 x 512 x 128: the largest band count it takes
    B, H, W = f.cube.shape
    cube = torch.as_tensor(f.cube, device="cuda")
    ref_v = torch.zeros(B, dtype=torch.float64, device="cuda")
    ref_l = torch.zeros(1, dtype=torch.float64, device="cuda")
    ref_I = hsc.hsc_pca_one_band(ctx, cube, eigvec=ref_v, eigval=ref_l)
    ctx.sync()
    stream = torch.cuda.Stream()
    outs = []
    for call in range(2):
        I = torch.full((H, W), -7.0, dtype=torch.float32, device="cuda")
        v = torch.zeros(B, dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = L.hsc_pca_one_band_noalloc(ctypes.c_void_p(stream.cuda_stream), cube.data_ptr(), B, H, W,
                                        hsc.HSC_PCA_MINMAX, I.data_ptr(), v.data_ptr(), lam.data_ptr())
        assert st == hsc.HSC_OK
        stream.synchronize()
        if call == 1:  # after the first call's one-time set-up nothing is allocated
            assert torch.cuda.mem_get_info()[0] >= free_before - (1 << 20)
        outs.append((I.cpu().numpy(), v.cpu().numpy(), float(lam.cpu()[0])))
    rI, rv, rl = ref_I.cpu().numpy(), ref_v.cpu().numpy(), float(ref_l.cpu()[0])
    for I, v, lam in outs:
        cos = float(v @ rv)
        assert cos > 0 and np.sqrt(max(0.0, 1 - cos * cos)) < V1_ANGLE
        assert lam == pytest.approx(rl, rel=1e-5)
        assert np.abs(I - rI).max() < I_TOL
    # the two calls in a row give the same answer
    np.testing.assert_array_equal(outs[0][0], outs[1][0])


def test_noalloc_rejects_sizes_beyond_its_scratch(hsc):
    import torch
    L = hsc.lib()
    B = hsc.HSC_NOALLOC_MAX_BANDS + 1
    cube = torch.zeros((B, 4, 4), dtype=torch.float32, device="cuda")
    I = torch.empty((4, 4), dtype=torch.float32, device="cuda")
    st = L.hsc_pca_one_band_noalloc(None, cube.data_ptr(), B, 4, 4, 1, I.data_ptr(), None, None)
    assert st == hsc.HSC_ERR_UNSUPPORTED
    st = L.hsc_pca_one_band_noalloc(None, None, 8, 4, 4, 1, I.data_ptr(), None, None)
    assert st == hsc.HSC_ERR_INVALID_ARG


def _offset_cube(torch, cube_np, offset_floats):
    """A device copy of the cube that starts offset_floats floats past a
    256-byte-aligned allocation (offset 1 = 4 bytes off the 16-byte grid)."""
    flat = torch.zeros(cube_np.size + offset_floats, dtype=torch.float32, device="cuda")
    view = flat[offset_floats:].view(cube_np.shape)
    view.copy_(torch.as_tensor(cube_np))
    torch.cuda.synchronize()
    return flat, view


@pytest.mark.parametrize("shape,offset", [((16, 7, 9), 1), ((64, 100, 120), 0),
                                          ((64, 100, 120), 1), ((125, 48, 52), 0)])
def test_noalloc_small_and_unaligned_cubes(hsc, ctx, shape, offset):
    """Frames that take the work-item or FP32-pipe Gram (too few pixels for
    64 partitions, a cube 4 bytes off the 16-byte grid, an odd pixel count)
    and band counts below 128: the fixed 64-partition scratch layout must
    give what the context entry point gives, twice in a row."""
    import torch
    L = hsc.lib()
    B, H, W = shape
    f = synth.make_frame(B * 13 + H, H, W, B, sigma=0.03)
    keep, cube = _offset_cube(torch, f.cube, offset)
    ref_v = torch.zeros(B, dtype=torch.float64, device="cuda")
    ref_l = torch.zeros(1, dtype=torch.float64, device="cuda")
    ref_I = hsc.hsc_pca_one_band(ctx, cube, eigvec=ref_v, eigval=ref_l)
    ctx.sync()
    rI, rv, rl = ref_I.cpu().numpy(), ref_v.cpu().numpy(), float(ref_l.cpu()[0])
    stream = torch.cuda.Stream()
    first = None
    for call in range(2):
        I = torch.full((H, W), -7.0, dtype=torch.float32, device="cuda")
        v = torch.zeros(B, dtype=torch.float64, device="cuda")
        lam = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = L.hsc_pca_one_band_noalloc(ctypes.c_void_p(stream.cuda_stream), cube.data_ptr(), B,
                                        H, W, hsc.HSC_PCA_MINMAX, I.data_ptr(), v.data_ptr(),
                                        lam.data_ptr())
        assert st == hsc.HSC_OK
        stream.synchronize()
        In, vn, ln = I.cpu().numpy(), v.cpu().numpy(), float(lam.cpu()[0])
        cos = float(vn @ rv)
        assert cos > 0 and np.sqrt(max(0.0, 1 - cos * cos)) < V1_ANGLE
        assert ln == pytest.approx(rl, rel=1e-5)
        assert np.abs(In - rI).max() < I_TOL
        if first is None:
            first = In
        else:  # the second call starts from the scratch the first one left
            np.testing.assert_array_equal(first, In)
    del keep
