"""Host side of the streaming sampler (no GPU): configuration parsing and
defaults, the per-batch draws and the flow-set schedule."""
import json

import numpy as np
import pytest

from paper_2512_09664_b300 import sampler as S

YAML = """
# a sampler configuration
image_shape: [256, 320]
batch_size: 8
flows_per_batch: 2      # B / F = 4 pairs per field
batches_per_flow: 3
seed: 11
seeding_density: [0.01, 0.05]
output: u8
flow:
  kind: fourier
  rms: 2.5
  grid: [128, 160]
jitter: {diameter: 0.1, intensity: 0.05}
hide_prob: 0.1
"""


def test_yaml_subset_parses_nested_mappings_lists_and_comments(tmp_path):
    p = tmp_path / "c.yaml"
    p.write_text(YAML)
    cfg = S.load_config(str(p))
    assert cfg["image_shape"] == [256, 320] and cfg["batch_size"] == 8
    assert cfg["flows_per_batch"] == 2 and cfg["batches_per_flow"] == 3
    assert cfg["flow"] == {"kind": "fourier", "rms": 2.5, "modes": 64, "min_wavelength": 16.0, "grid": [128, 160]}
    assert cfg["jitter"] == {"diameter": 0.1, "intensity": 0.05, "rho": 0.0}
    assert cfg["seeding_density"] == [0.01, 0.05] and cfg["output"] == "u8" and cfg["hide_prob"] == 0.1
    assert cfg["diameter"] == [1.0, 4.0]  # default


def test_json_and_dict_configs_agree(tmp_path):
    d = S.parse_yaml_subset(YAML)
    p = tmp_path / "c.json"
    p.write_text(json.dumps(d))
    assert S.load_config(str(p)) == S.load_config(d)


@pytest.mark.parametrize("bad", [{}, {"image_shape": [0, 8]}, {"image_shape": [8, 8], "flows_per_batch": 9,
                                                                  "batch_size": 4},
                                 {"image_shape": [8, 8], "batches_per_flow": 0},
                                 {"image_shape": [8, 8], "seeding_density": [0.2, 0.1]}])
def test_invalid_configs_rejected(bad):
    with pytest.raises(ValueError):
        S.load_config(bad)


def test_scalar_ranges_become_fixed_intervals():
    cfg = S.load_config({"image_shape": [8, 8], "seeding_density": 0.03, "rho": 0.5})
    assert cfg["seeding_density"] == [0.03, 0.03] and cfg["rho"] == [0.5, 0.5]


def test_descriptor_fast_path_matches_specs():
    # the sampler patches counts and pair ids into prebuilt descriptors: same bytes as building them anew
    import ctypes as C

    from paper_2512_09664_b300 import binding as B
    cfg = S.load_config(S.parse_yaml_subset(YAML))

    class Fake(S.Sampler):
        def __init__(self, cfg):  # descriptor part only, no device
            self.cfg, self.B, self.F = cfg, cfg["batch_size"], cfg["flows_per_batch"]
            self.H, self.W = cfg["image_shape"]
            self.gh, self.gw = cfg["flow"]["grid"]
            self.pairs = (B.PairDesc * self.B)()
    f = Fake(cfg)
    for k in (0, 7, 3):
        d = S.batch_densities(cfg, k)
        f._fill_pairs(d, k)
        ref = (B.PairDesc * f.B)()
        for b, spec in enumerate(S.batch_specs(cfg, d, k)):
            ref[b] = B.pair_desc(spec, b * 2 * f.H * f.W, spec.flow_index * f.gh * f.gw * 2, (f.gh, f.gw))
        assert C.string_at(C.addressof(f.pairs), C.sizeof(ref)) == C.string_at(C.addressof(ref), C.sizeof(ref))


def test_batch_draws_are_deterministic_and_in_range():
    cfg = S.load_config(S.parse_yaml_subset(YAML))
    a, b = S.batch_densities(cfg, 5), S.batch_densities(cfg, 5)
    assert np.array_equal(a, b) and not np.array_equal(a, S.batch_densities(cfg, 6))
    assert a.min() >= 0.01 and a.max() <= 0.05
    specs = S.batch_specs(cfg, a, 5)
    assert [p.pair_id for p in specs] == list(range(40, 48))  # batch 5 of 8 pairs
    assert [p.flow_index for p in specs] == [0, 0, 0, 0, 1, 1, 1, 1]
    assert [p.n_particles for p in specs] == [int(np.floor(x * 256 * 320)) for x in a]
    assert all(float(p.jitter_d) == np.float32(0.1) for p in specs)


def test_flow_sets_change_every_batches_per_flow():
    cfg = S.load_config(S.parse_yaml_subset(YAML))
    assert [S.flow_set_of(cfg, k) for k in range(8)] == [0, 0, 0, 1, 1, 1, 2, 2]
    from paper_2512_09664_b300 import workloads as W
    a = W.fourier_modes_set(S.flow_set_key(11, 0), 4, 256, 320)
    b = W.fourier_modes_set(S.flow_set_key(11, 1), 4, 256, 320)
    assert a.shape == (4, 64, 4) and not np.array_equal(a[..., 2], b[..., 2])
    assert len({tuple(a[f, :, 2]) for f in range(4)}) == 4  # the fields of a set differ
    # the spectrum of a set's fields is fourier_modes' spectrum
    one = W.fourier_modes(5, 256, 320)
    assert np.allclose(np.hypot(a[0, :, 0], a[0, :, 1]), np.hypot(one[:, 0], one[:, 1]))
    assert np.allclose(a[0, :, 3], one[:, 3])
