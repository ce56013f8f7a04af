"""The C ABI without a GPU: the library loads, exports what include/synthpix.h
declares, and rejects bad arguments with the documented status codes before
touching the device (these calls never reach CUDA)."""
import ctypes as C
import os
import re

import pytest

from paper_2512_09664_b300 import binding as B
from paper_2512_09664_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "synthpix.h")).read()
    return sorted(set(re.findall(r"\b(synthpix_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = B.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert L.synthpix_version() == 3


def test_descriptor_sizes_match_header():
    assert C.sizeof(B.PairDesc) == 160 and C.sizeof(B.BatchDesc) == 64


def _packed():
    return B.pack(W.batch_512_u8(n_pairs=2))


FAKE = C.c_void_p(0x7F0000000000)  # never dereferenced: validation fails first


def _render(pk, ws_bytes=1 << 30, ws=FAKE, flows=FAKE, images=FAKE):
    return B.lib().synthpix_render_pairs(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, flows, images,
                                         ws, ws_bytes, None)


@pytest.mark.parametrize("field,value", [
    ("out_dtype", 9), ("quant_bits", 0), ("integrator", 3), ("n_substeps", 0), ("n_substeps", 5000),
    ("dt", float("nan")), ("tile", 48), ("hide_prob", -0.1), ("hide_prob", 1.5), ("hide_prob", float("nan"))])
def test_bad_batch_fields_are_rejected(field, value):
    pk = _packed()
    setattr(pk.batch, field, value)
    assert _render(pk) == B.EINVAL
    assert B.last_error()
    assert B.lib().synthpix_workspace_bytes(C.byref(pk.batch), pk.pairs, pk.n_pairs) == 0


@pytest.mark.parametrize("field,value", [
    ("height", 0), ("width", 40000), ("flow_h", 0), ("flow_offset", -2), ("flow_offset", 3),
    ("d_min", 0.0), ("d_max", 40.0), ("d_dist", 2), ("i_min", 2.0), ("blur_sigma", 9.0),
    ("noise_sigma", -1.0), ("z_min", 5.0), ("sheet_sigma", float("inf")), ("dy_min", 2.0), ("dy_max", 40.0),
    ("dy_min", -1.0), ("rho_max", 0.99), ("rho_min", 0.5), ("jitter_d", -0.1), ("jitter_i", float("nan")),
    ("jitter_rho", -1.0)])
def test_bad_pair_fields_are_rejected(field, value):
    pk = _packed()
    setattr(pk.pairs[1], field, value)
    assert _render(pk) == B.EINVAL
    assert "pair 1" in B.last_error()


def test_reserved_fields_and_flags_unsupported():
    pk = _packed()
    pk.batch.flags = 8  # the first bit no flag uses
    assert _render(pk) == B.EUNSUPPORTED
    pk = _packed()
    pk.batch.reserved[0] = 1
    assert _render(pk) == B.EUNSUPPORTED


def test_workspace_checks():
    pk = _packed()
    pk.batch.tile = 32  # a fixed tile: workspace_bytes is then exactly what the render needs
    need = B.workspace_bytes(pk)
    assert need > 0
    assert _render(pk, ws_bytes=need - 1) == B.EWORKSPACE
    assert _render(pk, ws=None) == B.EWORKSPACE
    assert _render(pk, ws=C.c_void_p(0x7F0000000010)) == B.EWORKSPACE  # not 256-aligned


def test_null_and_misaligned_buffers():
    pk = _packed()
    assert _render(pk, flows=None) == B.EINVAL
    assert _render(pk, flows=C.c_void_p(0x7F0000000004)) == B.EINVAL
    assert _render(pk, images=None) == B.EINVAL
    assert B.lib().synthpix_render_pairs(None, pk.pairs, None, 2, FAKE, FAKE, FAKE, 1 << 30, None) == B.EINVAL
    assert B.lib().synthpix_render_pairs(C.byref(pk.batch), None, None, 2, FAKE, FAKE, FAKE, 1 << 30,
                                         None) == B.EINVAL
    assert B.lib().synthpix_render_pairs(C.byref(pk.batch), pk.pairs, None, -1, FAKE, FAKE, FAKE, 1 << 30,
                                         None) == B.EINVAL


def test_zero_pairs_is_a_no_op():
    pk = _packed()
    assert B.lib().synthpix_render_pairs(C.byref(pk.batch), pk.pairs, None, 0, None, None, None, 0,
                                         None) == B.OK


def test_auto_tile_workspace_covers_every_candidate():
    pk = _packed()
    auto = B.workspace_bytes(pk)
    for t in (16, 32, 64, 128):
        pk.batch.tile = t
        assert B.workspace_bytes(pk) <= auto


def test_workspace_grows_with_particles_and_tiles():
    small = B.workspace_bytes(B.pack(W.batch_512_u8(n_pairs=1)))
    big = B.workspace_bytes(B.pack(W.batch_512_u8(n_pairs=2)))
    assert big > small


def test_gather_advection_flag_accepted():
    pk = _packed()
    pk.batch.flags = B.FLAG_GATHER_ADVECT
    assert B.workspace_bytes(pk) > 0


def test_tiled_advection_flag_accepted_and_exclusive():
    pk = _packed()
    pk.batch.flags = B.FLAG_TILED_ADVECT
    assert B.workspace_bytes(pk) > 0
    pk.batch.flags = B.FLAG_TILED_ADVECT | B.FLAG_GATHER_ADVECT
    with pytest.raises(B.SynthpixError, match="exclude each other"):
        B.workspace_bytes(pk)


def test_advect_particles_rejects_missing_buffers():
    pk = _packed()
    L = B.lib()
    assert L.synthpix_advect_particles(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, None, FAKE, None, FAKE,
                                       1 << 30, None) == B.EINVAL
    assert L.synthpix_advect_particles(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, None, None, FAKE, FAKE,
                                       1 << 30, None) == B.EINVAL


def test_general_shape_fields_accepted_and_size_the_workspace():
    pk = _packed()
    base = B.workspace_bytes(pk)
    pk.batch.hide_prob = 0.25  # per-frame shapes: one float4 per particle and frame more
    hidden = B.workspace_bytes(pk)
    assert hidden > base
    pk.pairs[0].dy_min, pk.pairs[0].dy_max = 1.0, 3.0  # general shapes: 32-byte bin records
    pk.pairs[1].rho_min, pk.pairs[1].rho_max = -0.5, 0.5
    assert B.workspace_bytes(pk) > hidden
    assert _render(pk, ws_bytes=16) == B.EWORKSPACE  # validation passed up to the workspace check


def test_given_particles_and_adjoint_reject_shape_variation():
    pk = _packed()
    pk.pairs[0].jitter_i = 0.1
    L = B.lib()
    assert L.synthpix_render_pairs_from(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, FAKE, FAKE, FAKE, FAKE,
                                        1 << 30, None) == B.EUNSUPPORTED
    assert "round particles" in B.last_error()
    pk.batch.out_dtype = B.DTYPE_CODE["f32"]
    pk.batch.quant_bits = 0
    assert L.synthpix_render_backward(C.byref(pk.batch), pk.pairs, None, pk.n_pairs, None, FAKE, FAKE, FAKE,
                                      None, FAKE, 1 << 30, None) == B.EUNSUPPORTED
    assert "round particles" in B.last_error()


def test_histogram_matching_validation():
    pk = _packed()
    L = B.lib()
    assert L.synthpix_match_histogram_workspace_bytes(C.byref(pk.batch), pk.pairs, pk.n_pairs) > 0
    assert L.synthpix_match_histogram(C.byref(pk.batch), pk.pairs, pk.n_pairs, FAKE, FAKE, FAKE, 16, None) == \
        B.EWORKSPACE
    assert L.synthpix_match_histogram(C.byref(pk.batch), pk.pairs, pk.n_pairs, None, FAKE, FAKE, 1 << 30, None) == \
        B.EINVAL
    pk.batch.out_dtype, pk.batch.quant_bits = B.DTYPE_CODE["f32"], 0
    assert L.synthpix_match_histogram(C.byref(pk.batch), pk.pairs, pk.n_pairs, FAKE, FAKE, FAKE, 1 << 30, None) == \
        B.EUNSUPPORTED
    assert L.synthpix_match_histogram_workspace_bytes(C.byref(pk.batch), pk.pairs, pk.n_pairs) == 0


def test_binding_export_list_is_the_header():
    assert sorted(B.exported_symbols()) == _declared()


def test_alu_probe_validation_before_any_launch():
    # the probes live in a measurement library of their own, not in the renderer's ABI
    from paper_2512_09664_b300 import measure
    assert not hasattr(B.lib(), "synthpix_alu_probe")
    L = measure.lib()
    ops = C.c_int64(-1)
    sink = C.c_void_p(256)  # never dereferenced: every call below fails its argument checks first
    assert L.synthpix_alu_probe(4, 16, sink, 1 << 20, C.byref(ops), None) == measure.EINVAL
    assert L.synthpix_alu_probe(-1, 16, sink, 1 << 20, C.byref(ops), None) == measure.EINVAL
    assert L.synthpix_alu_probe(0, 0, sink, 1 << 20, C.byref(ops), None) == measure.EINVAL
    assert L.synthpix_alu_probe(0, (1 << 16) + 1, sink, 1 << 20, C.byref(ops), None) == measure.EINVAL
    assert L.synthpix_alu_probe(0, 16, sink, 1 << 20, None, None) == measure.EINVAL
    assert L.synthpix_alu_probe(0, 16, None, 1 << 20, C.byref(ops), None) == measure.EINVAL
    assert L.synthpix_alu_probe(0, 16, C.c_void_p(258), 1 << 20, C.byref(ops), None) == measure.EINVAL
    assert ops.value == -1
    assert "alu probe" in measure.last_error()


def test_pack_keeps_flow_grids_on_even_floats_with_odd_w_grids():
    # 3 x 5 nodes: an odd w grid after the first flow grid must not shift the
    # second grid onto an odd float (its float2 nodes need 8-byte alignment)
    import numpy as np
    flows = [W.fourier_flow(3, 5, 20, 24, rms=1.0, seed=1), W.fourier_flow(3, 5, 20, 24, rms=1.0, seed=2)]
    pairs = [W.PairSpec(height=20, width=24, n_particles=10, pair_id=b, flow_index=b) for b in range(2)]
    wl = W.Workload(name="w", seed=3, pairs=pairs, flows=flows,
                    flows_w=[np.full((3, 5), 0.1, np.float32), np.full((3, 5), -0.1, np.float32)])
    pk = B.pack(wl)
    assert [pk.pairs[b].flow_offset % 2 for b in range(2)] == [0, 0]
    assert pk.pairs[1].flow_offset >= 2 * 15 + 15
    assert B.workspace_bytes(pk) > 0
