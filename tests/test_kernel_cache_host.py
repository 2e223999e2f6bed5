"""The kernel-set cache key (aw_kernel_spec_hash), host only: it equals the
FNV-1a 64 of the canonical little-endian spec encoding the header documents
(re-encoded here with struct), is stable, and changes with every field and
array entry that defines the tables."""
import math
import struct

import numpy as np
import pytest

from paper_2206_15117_gb300 import aw

BASE = dict(N=256, dl=math.radians(3.0) / 256, OS=8, W=7.0, npol=4, nw=3, w_max=900.0, supports=[16, 20, 24],
            pa=[0.1, -0.4], fbin_freqs=[1.3e9, 1.4e9], dish_d=12.0, d_xy=0.01 * np.exp(0.4j),
            d_yx=0.01 * np.exp(-1.3j), eps=0.2, role=aw.AW_ROLE_GRID, storage=aw.AW_STORAGE_FP32,
            point_l=0.0, point_m=0.0)


def _fnv(b: bytes) -> int:
    h = 1469598103934665603
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _encode(s, type_leak=()):
    i32 = lambda v: struct.pack("<i", int(v))
    f64 = lambda v: struct.pack("<d", float(v))
    b = i32(s["N"]) + f64(s["dl"]) + i32(s["OS"]) + f64(s["W"]) + i32(s["npol"]) + i32(s["nw"]) + f64(s["w_max"])
    b += b"".join(i32(x) for x in s["supports"])
    b += i32(len(s["pa"])) + b"".join(f64(x) for x in s["pa"])
    b += i32(len(s["fbin_freqs"])) + b"".join(f64(x) for x in s["fbin_freqs"])
    b += f64(s["dish_d"]) + f64(complex(s["d_xy"]).real) + f64(complex(s["d_xy"]).imag)
    b += f64(complex(s["d_yx"]).real) + f64(complex(s["d_yx"]).imag) + f64(s["eps"])
    b += i32(s["role"]) + i32(s["storage"]) + f64(s["point_l"]) + f64(s["point_m"])
    b += i32(max(1, len(type_leak)))   # normalised: 0 and 1 type both mean baseline-averaged kernels
    if len(type_leak) >= 2:
        for dxy, dyx in type_leak:
            b += f64(complex(dxy).real) + f64(complex(dxy).imag) + f64(complex(dyx).real) + f64(complex(dyx).imag)
    return b


def test_hash_is_the_documented_encoding():
    assert aw.aw_kernel_spec_hash(**BASE) == _fnv(_encode(BASE))
    tl = [(0.01, 0.02j), (-0.01j, 0.03)]
    assert aw.aw_kernel_spec_hash(**BASE, type_leak=tl) == _fnv(_encode(BASE, tl))


@pytest.mark.parametrize("field,value", [
    ("N", 512), ("dl", BASE["dl"] * 1.0000001), ("OS", 4), ("W", 6.0), ("nw", 2), ("w_max", 901.0),
    ("supports", [16, 20, 26]), ("pa", [0.1, -0.41]), ("fbin_freqs", [1.3e9, 1.41e9]), ("dish_d", 13.0),
    ("d_xy", 0.011 * np.exp(0.4j)), ("d_yx", 0.01 * np.exp(-1.2j)), ("eps", 0.21), ("role", aw.AW_ROLE_DEGRID),
    ("storage", aw.AW_STORAGE_BF16), ("point_l", 0.001), ("point_m", -0.001)])
def test_hash_changes_with_every_field(field, value):
    spec = dict(BASE, **{field: value})
    if field == "nw":
        spec["supports"] = spec["supports"][:2]
    assert aw.aw_kernel_spec_hash(**spec) != aw.aw_kernel_spec_hash(**BASE)


def test_hash_is_stable_and_validates():
    assert aw.aw_kernel_spec_hash(**BASE) == aw.aw_kernel_spec_hash(**dict(BASE))
    assert aw.aw_kernel_spec_hash(**BASE, type_leak=[(0.01, 0.0), (0.02, 0.0)]) != aw.aw_kernel_spec_hash(**BASE)
    with pytest.raises(aw.AWError):
        aw.aw_kernel_spec_hash(**dict(BASE, N=300))
