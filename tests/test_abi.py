"""Host-side checks of the C ABI: the library loads, exports every function declared in
include/dg.h, computes its LGL basis without a GPU, and refuses to run without one."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    import paper_2511_17551_gb300 as dg
    lib = dg.lib()
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(dg.EXPORTED), set(declared) - set(dg.EXPORTED)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_library_lgl_matches_oracle(orc, N):
    import paper_2511_17551_gb300 as dg
    x, w = dg.dg_lgl_nodes(N)
    xo, wo = orc.lgl(N)
    assert np.allclose(x, xo, atol=1e-15) and np.allclose(w, wo, atol=1e-15)


def test_no_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2511_17551_gb300 as dg
    import workloads as W
    x, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face = W.box_mesh((2, 2, 2), x, (0, 0, 0), (1, 1, 1))
    with pytest.raises(dg.DgError) as ei:
        dg.Solver(3, 3, xyz, nbr, face)
    assert ei.value.code == dg.DG_ECUDA
