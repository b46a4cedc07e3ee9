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


def test_invalid_descriptors_rejected_before_any_device_use():
    """Argument validation precedes every device call: an empty mesh, an unsupported degree,
    a neighbour out of range and out-of-range options return DG_EINVAL here too."""
    import paper_2511_17551_gb300 as dg
    import workloads as W
    x, _ = dg.dg_lgl_nodes(3)
    xyz, nbr, face = W.box_mesh((2, 2, 2), x, (0, 0, 0), (1, 1, 1))
    bad_nbr = nbr.copy()
    bad_nbr[0, 0] = 8
    cases_ = [
        dict(xyz=xyz[:0], nbr=nbr[:0], face=face[:0], N=3, kw={}),            # K = 0
        dict(xyz=xyz, nbr=nbr, face=face, N=6, kw={}),                         # degree not built
        dict(xyz=xyz, nbr=bad_nbr, face=face, N=3, kw={}),                     # neighbour >= K
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(volume_flux=6)),
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(surface_flux=-1)),
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(sutherland_s=-0.1)),
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(sutherland_s=0.4, sutherland_rt=0.0)),
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(indicator_variable=2)),
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(positivity_eps=-1.0)),
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(alpha_max=1.5)),
        dict(xyz=xyz, nbr=nbr, face=face, N=3, kw=dict(equations=1, mu=0.0)),
    ]
    for c in cases_:
        with pytest.raises(dg.DgError) as ei:
            dg.Solver(3, c["N"], c["xyz"], c["nbr"], c["face"], **c["kw"])
        assert ei.value.code == dg.DG_EINVAL, c["kw"]
