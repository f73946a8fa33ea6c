"""Seeded synthetic inputs (volumes, transfer functions, edit sequences).

Shared by the CPU oracle's tests, the CUDA path's tests and the benchmark; holds none of
the method's arithmetic.  Workload recipes:

* tiny  : 128^3 uint8, 4^3 blocks (32^3 grid), K=16, N=256, 100 TF edits (seed 0)
* ct    : 512^3 12-bit uint16, 4^3 blocks (128^3 grid), K=32, N=4096, 1000 edits (seed 1)
* large : 1024x1024x1795 12-bit uint16, 4^3 blocks (256x256x449 grid), K=64, N=4096 (seed 2)
* batch : 64 volumes, sides U[64, 384], alternating uint8 / 12-bit, K alternating 16 / 32,
          one TF edit each (seed 4)
"""
from .volumes import (tiny_volume, ct_volume, large_volume, as_numpy, volume_sha256,  # noqa: F401
                      volume_of, batch_specs)
from .tfs import (tf_edit_sequence, zero_tf, all_visible_tf, single_intensity_tf,  # noqa: F401
                  aligned_tf, special_tfs, uniform_borders, tf_from_ramps, Ramp)

WORKLOADS = {
    "tiny": dict(dims=(128, 128, 128), dtype="u8", block=4, apron=1, K=16, N=256,
                 edits=100, seed=0),
    "ct": dict(dims=(512, 512, 512), dtype="u16", block=4, apron=1, K=32, N=4096,
               edits=1000, seed=1),
    "large": dict(dims=(1024, 1024, 1795), dtype="u16", block=4, apron=1, K=64, N=4096,
                  edits=1000, seed=2),
    # the large recipe cut to 448 slices: a profiling size (about 1.5 GB on the device)
    "mid": dict(dims=(1024, 1024, 448), dtype="u16", block=4, apron=1, K=64, N=4096,
                edits=1000, seed=2),
}


def make_volume(name: str, device="cpu"):
    w = WORKLOADS[name]
    if name == "tiny":
        return tiny_volume(w["seed"], device=device)
    if name == "ct":
        return ct_volume(w["seed"], device=device)
    if name in ("large", "mid"):
        return large_volume(w["seed"], dims=w["dims"], device=device)
    raise KeyError(name)
