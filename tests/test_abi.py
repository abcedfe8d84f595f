"""The C ABI library: it loads, exports every function include/xpinn.h
declares, matches the binding's structure layout, and rejects invalid
problem descriptions on the host (before any CUDA call), so these run
without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2104_10013_gb300 import build as B
from paper_2104_10013_gb300 import problems as P
from paper_2104_10013_gb300 import xpinn as X

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xpinn.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return X.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xpinn_\w+)\s*\(", src)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    src = open(os.path.join(ROOT, "paper_2104_10013_gb300", "xpinn.py")).read()
    for n in declared_functions():
        assert f'"{n}"' in src, n


def test_header_constants_match_binding():
    src = open(HEADER).read()
    get = lambda name: int(re.search(rf"#define {name} (\d+)", src).group(1))
    assert get("XPINN_MAX_NETS") == X.MAX_NETS
    assert get("XPINN_MAX_LAYERS") == X.MAX_LAYERS
    assert get("XPINN_N_TERMS") == X.N_TERMS == P.N_TERMS


def test_struct_layout_is_plain_c():
    # sizes the C compiler gives the header structs (compiled here with gcc)
    code = r'''
#include <stdio.h>
#include <stddef.h>
#include "xpinn.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(xpinn_net_desc), sizeof(xpinn_subdomain_desc),
         sizeof(xpinn_interface_desc), sizeof(xpinn_problem_desc), sizeof(xpinn_options),
         offsetof(xpinn_subdomain_desc, lr));
  return 0;
}
'''
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(code)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        got = list(map(int, subprocess.run([exe], capture_output=True, text=True).stdout.split()))
    want = [C.sizeof(X.NetDesc), C.sizeof(X.SubDesc), C.sizeof(X.IfaceDesc), C.sizeof(X.ProblemDesc),
            C.sizeof(X.Options), X.SubDesc.lr.offset]
    assert got == want


def _create(lib, pb, mutate=None):
    """Build a description like Solver does, let `mutate` break it, call create."""
    s = X.Solver.__new__(X.Solver)
    keep = []

    def arr(a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        keep.append(a)
        return a.ctypes.data
    subs = (X.SubDesc * pb.n_sub)()
    for q, sd in enumerate(pb.subs):
        d = subs[q]
        d.n_nets = len(sd.nets)
        for n, net in enumerate(sd.nets):
            d.nets[n].n_layers = len(net.widths) - 1
            for k, w in enumerate(net.widths):
                d.nets[n].widths[k] = w
        d.n_res = sd.res_xy.shape[0]
        d.res_xy = arr(sd.res_xy)
        d.res_f = arr(sd.res_f)
        d.lr = sd.lr
        d.w_res = d.w_avg = d.w_iface = 1.0
    ifs = (X.IfaceDesc * max(1, len(pb.ifaces)))()
    for e, it in enumerate(pb.ifaces):
        ifs[e].q, ifs[e].q_plus, ifs[e].method = it.q, it.qp, it.method
        ifs[e].n_pts = it.xy.shape[0]
        ifs[e].xy = arr(it.xy)
    desc = X.ProblemDesc()
    desc.pde, desc.nu, desc.re = pb.pde, pb.nu, 1.0
    desc.n_sub, desc.subs = pb.n_sub, subs
    desc.n_iface, desc.ifaces = len(pb.ifaces), ifs
    desc.beta1, desc.beta2, desc.eps = 0.9, 0.999, 1e-8
    desc.init_params = arr(pb.packed_params())
    if mutate:
        mutate(desc, subs, ifs)
    h = C.c_void_p()
    rc = lib.xpinn_create(C.byref(desc), C.byref(h))
    return rc, lib.xpinn_last_error().decode(), h


@pytest.mark.parametrize("name,mutate,code", [
    ("pde", lambda d, s, f: setattr(d, "pde", 9), -1),
    ("no subdomains", lambda d, s, f: setattr(d, "n_sub", 0), -1),
    ("no params", lambda d, s, f: setattr(d, "init_params", None), -1),
    ("beta", lambda d, s, f: setattr(d, "beta2", 1.5), -1),
    ("input width", lambda d, s, f: s[0].nets[0].widths.__setitem__(0, 3), -1),
    ("too deep", lambda d, s, f: setattr(s[0].nets[0], "n_layers", 13), -6),
    ("too wide", lambda d, s, f: s[0].nets[0].widths.__setitem__(1, 500), -6),
    ("outputs", lambda d, s, f: s[0].nets[0].widths.__setitem__(4, 2), -1),
    ("two nets for burgers", lambda d, s, f: setattr(s[0], "n_nets", 2), -1),
    ("interface self", lambda d, s, f: setattr(f[0], "q_plus", f[0].q), -1),
    ("interface range", lambda d, s, f: setattr(f[0], "q_plus", 99), -1),
    ("method", lambda d, s, f: setattr(f[0], "method", 7), -1),
    ("negative points", lambda d, s, f: setattr(s[1], "n_res", -5), -1),
    ("models", lambda d, s, f: setattr(d, "subs_per_model", 3), -1),
])
def test_invalid_descriptions_are_rejected_on_the_host(lib, name, mutate, code):
    pb = P.burgers_cpinn(n_res=16, n_iface=4, n_bc=4)
    rc, msg, h = _create(lib, pb, mutate)
    assert rc == code, (name, rc, msg)
    assert msg
    assert not h.value


def test_nonfinite_inputs_are_rejected(lib):
    pb = P.burgers_cpinn(n_res=16, n_iface=4, n_bc=4)
    pb.subs[2].res_xy[3, 1] = np.nan
    rc, msg, _ = _create(lib, pb)
    assert rc == -1 and "finite" in msg


def test_null_handles_are_errors_not_crashes(lib):
    assert lib.xpinn_destroy(None) == 0
    assert lib.xpinn_grad(None, None, None, None) == -1
    assert lib.xpinn_step(None, 1, None, None) == -1
    assert lib.xpinn_num_params(None) == -1
    assert lib.xpinn_last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library the binding raises, and so
    does every entry point that needs it."""
    from paper_2104_10013_gb300 import problems as P
    from paper_2104_10013_gb300 import xpinn as X
    from tests.cases import tiny_problem
    monkeypatch.setattr(X, "_LIB", None)
    monkeypatch.setattr(X, "lib_path", lambda: str(tmp_path / "libxpinn.so"))
    with pytest.raises(RuntimeError, match="not built"):
        X.load()
    with pytest.raises(RuntimeError, match="not built"):
        X.Solver(tiny_problem(P.PDE_POISSON, P.XPINN))
