"""The no-allocation entry point, synthpix_render_pairs_noalloc.

It serves callers that cannot allocate device memory (hosts that own all
device memory through their own allocator, fixed-budget runtimes, loops that
cannot afford cudaMalloc's synchronisation): they pass only inputs and
outputs, and the render's scratch lives in a fixed array inside the library.
These tests call it through the C ABI and check it against the workspace
entry point, synthpix_render_pairs.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2512_09664_b300 import binding as B
from paper_2512_09664_b300 import workloads as W

SCRATCH_BYTES = 32 << 20
FAKE = C.c_void_p(0x7F0000000000)  # never dereferenced: rejected before any device call


def _fn():
    L = B.lib()
    f = L.synthpix_render_pairs_noalloc
    f.argtypes = [C.POINTER(B.BatchDesc), C.POINTER(B.PairDesc), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                  C.c_void_p]
    f.restype = C.c_int
    return f


def test_noalloc_rejects_batches_larger_than_its_scratch():
    pk = B.pack(W.batch_512_u8(n_pairs=64))
    assert B.workspace_bytes(pk) > SCRATCH_BYTES
    rc = _fn()(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, FAKE, FAKE, None)
    assert rc == B.EWORKSPACE
    assert "scratch" in B.last_error()
    # invalid descriptors keep their own status code
    pk.batch.n_substeps = 0
    assert _fn()(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, FAKE, FAKE, None) == B.EINVAL


def test_noalloc_sizes_its_check_from_the_tile_the_render_runs():
    # tile 0: synthpix_workspace_bytes covers every edge the autotuner tries
    # (tile 16 has the most bin counters), more than the 32 MiB array; the
    # render itself runs the default edge (128 at 512 x 512), which fits.  The
    # size check must pass; without a GPU the call then stops at the device
    # query, never at the size check.
    import torch
    pk = B.pack(W.batch_512_u8(n_pairs=4))
    assert pk.batch.tile == 0
    assert B.workspace_bytes(pk) > SCRATCH_BYTES
    assert B.workspace_bytes(B.pack(W.batch_512_u8(n_pairs=4), tile=128)) <= SCRATCH_BYTES
    if torch.cuda.is_available():
        pytest.skip("checks the size decision without launching; a GPU would render here")
    rc = _fn()(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, FAKE, FAKE, None)
    assert rc == B.ECUDA and "scratch" not in B.last_error()


def test_noalloc_reports_invalid_descriptors_with_the_plans_message():
    pk = B.pack(W.batch_512_u8(n_pairs=2))
    pk.pairs[1].d_min = -1.0
    rc = _fn()(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, FAKE, FAKE, None)
    assert rc == B.EINVAL
    msg = B.last_error()
    assert "pair 1" in msg and "workspace" not in msg


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    # two different batches back to back: the second call runs on scratch
    # that still holds the first call's contents
    first = W.batch_512_u8(n_pairs=3)
    second = W.uneven_batch(n_pairs=5, sizes=(64, 128, 256))
    for wl in (first, second):
        ref = B.Renderer(wl)
        # the render's own plan fits the array (the no-allocation call checks it
        # and returns SYNTHPIX_EWORKSPACE otherwise); the tile-0 workspace bound
        # that synthpix_workspace_bytes reports may be larger
        assert B.workspace_bytes(B.pack(wl, tile=128 if wl is first else 64)) <= SCRATCH_BYTES
        ref.render()
        out = torch.zeros_like(ref.images)
        stream = torch.cuda.current_stream()
        rc = _fn()(C.byref(ref.pk.batch), ref.pk.pairs, None, ref.pk.n_pairs, C.c_void_p(ref.flows.data_ptr()),
                   C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == B.OK, B.last_error()
        torch.cuda.synchronize()
        if out.dtype == torch.uint16:
            a = out.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.int64)
            b = ref.images.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.int64)
        else:
            a = out.cpu().numpy().astype(np.int64)
            b = ref.images.cpu().numpy().astype(np.int64)
        # quantised codes: the tests' tolerance for codes away from rounding
        # boundaries is zero, and both calls run the same kernels
        assert np.array_equal(a, b)
