"""The allocation-free inpainting entry point (hdi_inpaint_noalloc).

Some callers cannot allocate device memory while they run (code inside a
CUDA stream capture, loops with a fixed memory plan, processes whose device
allocator belongs to another runtime). hdi_inpaint_noalloc serves them from
a statically declared device array instead of a context workspace. These
tests call it through the C ABI and check it against hdi_inpaint on two
calls in a row with different images, masks and sizes, so that contents
left in the shared array by the first call cannot leak into the second.
The file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

from gpu_util import torch, need_gpu, ctx, dev
from synthdata import synth_image, synth_rgb, random_mask

pytestmark = pytest.mark.gpu


def noalloc_fn():
    import paper_2401_06747_b300 as hdi
    lib = hdi.load()
    fn = lib.hdi_inpaint_noalloc
    P = ctypes.POINTER
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, P(hdi.Image), P(hdi.Mask), P(hdi.Image), ctypes.c_double,
                   P(hdi.Stats)]
    fn.restype = ctypes.c_int
    return fn, hdi


def solve_both(f, c, tol):
    fn, hdi = noalloc_fn()
    fd, cd = dev(f), dev(c)
    ref = torch.empty_like(fd)
    ctx().inpaint(fd, cd, ref, tol=tol)
    out = torch.full_like(fd, float("nan"))
    st = hdi.Stats()
    stream = torch.cuda.current_stream().cuda_stream
    rc = fn(0, ctypes.c_void_p(stream), ctypes.byref(hdi.image_of(fd)), ctypes.byref(hdi.mask_of(cd)),
            ctypes.byref(hdi.image_of(out)), tol, ctypes.byref(st))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy(), ref.cpu().numpy(), st


def test_matches_hdi_inpaint_on_two_calls_in_a_row():
    need_gpu()
    # first call: RGB FP32, 4% mask
    f1 = synth_rgb(200, 150, seeds=(31, 32, 33), dtype=np.float32)
    c1 = random_mask(200, 150, 0.04, 34)
    rc, out, ref, st = solve_both(f1, c1, 1e-6)
    assert rc == 0 and st.rel_res <= 1e-6
    assert np.abs(out - ref).max() <= 1e-3
    # second call: a smaller grey FP64 image with a different mask density
    f2 = synth_image(96, 128, 35)
    c2 = random_mask(96, 128, 0.08, 36)
    rc, out, ref, st = solve_both(f2, c2, 1e-8)
    assert rc == 0 and st.rel_res <= 1e-8
    assert np.abs(out - ref).max() <= 1e-6


def test_rejects_images_beyond_the_static_scratch():
    need_gpu()
    fn, hdi = noalloc_fn()
    f = torch.zeros((3, 1024, 1024), dtype=torch.float32, device="cuda")
    c = torch.ones((1024, 1024), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(f)
    rc = fn(0, None, ctypes.byref(hdi.image_of(f)), ctypes.byref(hdi.mask_of(c)), ctypes.byref(hdi.image_of(out)),
            1e-6, None)
    assert rc == -1
    # host buffers would need staging memory and are refused as well
    fh = np.zeros((1, 16, 16), np.float32)
    ch = np.ones((16, 16), np.uint8)
    oh = np.zeros_like(fh)
    rc = fn(0, None, ctypes.byref(hdi.image_of(fh)), ctypes.byref(hdi.mask_of(ch)), ctypes.byref(hdi.image_of(oh)),
            1e-6, None)
    assert rc == -1
