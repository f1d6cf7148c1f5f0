"""C ABI: the library loads, exports every declared symbol, and rejects
malformed input on the host before any device call (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import rvegen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "rve.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rve_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def rve():
    import __graft_entry__ as g
    g.build()
    import paper_2306_09427_gb300 as rve
    return rve


def test_exports_every_declared_symbol(rve):
    names = _declared()
    assert "rve_solve" in names and "rve_batch_create" in names and "rve_tangent" in names
    for n in names:
        assert hasattr(rve.lib, n), n


def test_binding_uses_the_c_names(rve):
    for n in _declared():
        assert hasattr(rve, n), n


def test_options_default(rve):
    import ctypes
    o = rve._lib.rve_options()
    rve.rve_options_default(ctypes.byref(o))
    assert o.tol == 3e-7 and o.sigma_tol == 0.0 and o.max_iter == 200000 and o.check_every == 50
    assert o.precision == rve.RVE_PREC_MIXED and o.warm_start == 0 and o.threads == 0


def _packed():
    nets, F = rvegen.config_uniform(2, side=4)
    return rvegen.pack(nets)


@pytest.mark.parametrize("mutate,msg", [
    (lambda p: p.conn.__setitem__(0, p.conn[1]), "itself"),
    (lambda p: p.conn.__setitem__(0, 999), "out of range"),
    (lambda p: p.L0.__setitem__(3, 0.0), "rest length"),
    (lambda p: p.EA.__setitem__(3, -1.0), "EA"),
    (lambda p: p.B.__setitem__(3, -1.0), "B must"),
    (lambda p: p.B.__setitem__(3, np.nan), "B must"),
    (lambda p: p.X.__setitem__(5, np.inf), "non-finite"),
    (lambda p: p.node_off.__setitem__(1, p.node_off[2] + 1), "decreases"),
    (lambda p: p.is_boundary.__setitem__(slice(0, int(p.node_off[1])), 0), "no boundary"),
    (lambda p: p.V0.__setitem__(0, 0.0), "V0"),
])
def test_malformed_inputs_rejected_on_host(rve, mutate, msg):
    p = _packed()
    mutate(p)
    with pytest.raises(rve.RveError) as e:
        rve.RveBatch(p)
    assert e.value.code == rve.RVE_EINVAL
    assert msg in str(e.value)


def test_unknown_option_name_rejected(rve):
    with pytest.raises(TypeError):
        rve.RveBatch(_packed(), damping_scal=0.7)


def test_bad_options_rejected(rve):
    for kw in (dict(tol=0.0), dict(check_every=0), dict(precision=7), dict(threads=100), dict(warm_start=3),
               dict(damping_mode=2), dict(damping_mode=1, precision=0), dict(damping_scale=1.5),
               dict(damping_scale=-0.1)):
        with pytest.raises(rve.RveError) as e:
            rve.RveBatch(_packed(), **kw)
        assert e.value.code == rve.RVE_EINVAL
