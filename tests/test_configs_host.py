"""The five configurations' kernel specs (synthetic.config_spec) pass the
library's own spec validation (host only, through aw_kernel_spec_hash) and
have the shapes the configurations state."""
import numpy as np
import pytest

from paper_2206_15117_gb300 import aw
from paper_2206_15117_gb300 import synthetic as sy


@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5])
def test_config_specs_are_valid(cfg):
    src = 2 if cfg == 4 else cfg          # configuration 4 is configuration 2's inputs
    ob = sy.observation(src, time_samples=20) if src in (1, 3) else sy.observation(src, vis_fraction=0.001)
    kw = sy.config_spec(cfg, ob)
    h = aw.aw_kernel_spec_hash(**kw)
    assert h == aw.aw_kernel_spec_hash(**kw)
    N = {1: 512, 2: 2048, 3: 4096, 4: 2048, 5: 2048}[cfg]
    assert kw["N"] == N
    if cfg == 1:
        assert kw["npol"] == 1 and kw["supports"] == [7]
    elif cfg in (2, 4):
        assert kw["npol"] == 1 and kw["nw"] == 32 and min(kw["supports"]) == 8 and max(kw["supports"]) == 64
    else:
        assert kw["npol"] == 4 and kw["nw"] == 32 and len(kw["pa"]) >= 1 and len(kw["fbin_freqs"]) >= 1
        assert abs(abs(kw["d_xy"]) - 0.01) < 1e-12 and kw["eps"] == 0.2
        assert max(kw["supports"]) == (72 if cfg == 3 else 64)
    if cfg == 4:
        for st in (aw.AW_STORAGE_BF16, aw.AW_STORAGE_FP16):
            assert aw.aw_kernel_spec_hash(**kw, storage=st) != h
