"""The allocation-free inpainting entry point (hdi_inpaint_noalloc).

Some callers cannot allocate device memory while they run (a real-time loop
with a fixed memory plan, a process whose GPU memory belongs to another
runtime's allocator). hdi_inpaint_noalloc serves them from a statically
declared device array instead of a context workspace. These tests call it
through the C ABI and check it against hdi_inpaint on two calls in a row
with different images, masks and sizes, so that contents left in the shared
array by the first call cannot leak into the second; near its size limit
(400x400 RGB fits, 440x440 RGB does not); on a side stream; and that it
puts the caller's current device back. The file is named to be collected
last.
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


def solve_both(f, c, tol, stream=None):
    fn, hdi = noalloc_fn()
    fd, cd = dev(f), dev(c)
    ref = torch.empty_like(fd)
    ctx().inpaint(fd, cd, ref, tol=tol)
    torch.cuda.synchronize()
    out = torch.full_like(fd, float("nan"))
    st = hdi.Stats()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = fn(0, ctypes.c_void_p(s.cuda_stream), ctypes.byref(hdi.image_of(fd)), ctypes.byref(hdi.mask_of(cd)),
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


def test_just_under_the_size_limit_and_on_a_side_stream():
    """400x400 RGB (480,000 values) fits the 24 MiB array; the call runs on
    a stream other than the current one."""
    need_gpu()
    f = synth_rgb(400, 400, seeds=(41, 42, 43), dtype=np.float32)
    c = random_mask(400, 400, 0.05, 44)
    side = torch.cuda.Stream()
    rc, out, ref, st = solve_both(f, c, 1e-6, stream=side)
    assert rc == 0 and st.rel_res <= 1e-6
    assert np.abs(out - ref).max() <= 1e-3


def test_just_over_the_size_limit_is_refused():
    """440x440 RGB (580,800 values) needs more than the 24 MiB array."""
    need_gpu()
    fn, hdi = noalloc_fn()
    f = torch.zeros((3, 440, 440), dtype=torch.float32, device="cuda")
    c = torch.ones((440, 440), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(f)
    rc = fn(0, None, ctypes.byref(hdi.image_of(f)), ctypes.byref(hdi.mask_of(c)), ctypes.byref(hdi.image_of(out)),
            1e-6, None)
    assert rc == -1


def test_restores_the_callers_current_device():
    need_gpu()
    fn, hdi = noalloc_fn()
    lib = hdi.load()
    f = dev(synth_image(32, 48, 45).astype(np.float32)[None])
    c = dev(random_mask(32, 48, 0.1, 46))
    out = torch.empty_like(f)
    before = torch.cuda.current_device()
    rc = fn(0, None, ctypes.byref(hdi.image_of(f)), ctypes.byref(hdi.mask_of(c)), ctypes.byref(hdi.image_of(out)),
            1e-6, None)
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.cuda.current_device() == before
    # an out-of-range device index is refused before any device is touched
    rc = fn(1 << 20, None, ctypes.byref(hdi.image_of(f)), ctypes.byref(hdi.mask_of(c)),
            ctypes.byref(hdi.image_of(out)), 1e-6, None)
    assert rc == -1
    assert lib is not None
