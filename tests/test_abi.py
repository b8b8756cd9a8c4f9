"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every symbol that include/lbgb.h declares, and the
Python mirror of lb_params has the C layout."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbgb.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2004_04080_gb300 import build, lbgb

    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(lbgb.EXPORTS) == syms


def test_params_struct_layout_matches_c():
    from paper_2004_04080_gb300.lbgb import LbParams

    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "lbgb.h"
#define O(f) printf("%s %zu\n", #f, offsetof(lb_params, f));
int main(void) { printf("size %zu\n", sizeof(lb_params));
O(tau) O(G) O(zeta) O(rho0) O(bc) O(wall_u_lo) O(wall_u_hi) O(body_force) O(hertz_K)
O(hertz_sigma) O(hertz_rcap) O(lub_on) O(lub_hn) O(lub_hmin) O(lub_scale) O(side_wall_k)
O(side_wall_d) O(rotate) O(janus) O(janus_theta0) O(janus_width) O(rcut) O(delr) O(open) O(open_rho) O(open_extrap) return 0; }
'''
    tmp = os.path.join(ROOT, "paper_2004_04080_gb300", "_build")
    os.makedirs(tmp, exist_ok=True)
    c = os.path.join(tmp, "layout_check.c")
    exe = os.path.join(tmp, "layout_check")
    open(c, "w").write(prog)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict(l.split() for l in out if l)
    assert int(vals["size"]) == ctypes.sizeof(LbParams)
    for name, _ in LbParams._fields_:
        assert int(vals[name]) == getattr(LbParams, name).offset, name


def test_workspace_size_host_logic():
    from paper_2004_04080_gb300 import lbgb

    b32 = lbgb.lb_workspace_bytes(32, 32, 32, lbgb.LB_FP32, 4)
    b64 = lbgb.lb_workspace_bytes(32, 32, 32, lbgb.LB_FP64, 4)
    b16 = lbgb.lb_workspace_bytes(32, 32, 32, lbgb.LB_FP16, 4)
    N = 32 ** 3
    # two population buffers of 2 x 19 values per site dominate
    assert b64 > 2 * 38 * 8 * N and b32 > 2 * 38 * 4 * N and b16 > 38 * 2 * N
    assert b16 < b32 < b64
    for bad in [(0, 32, 32, 1, 0), (32, 32, 32, 7, 0), (32, 32, 3, 1, 0), (32, 32, 32, 1, -1)]:
        with pytest.raises(lbgb.LBError):
            lbgb.lb_workspace_bytes(*bad)
    # one component: 19 values per site in each buffer, no per-site coupling
    # arrays, and no particles
    one = lbgb.lb_workspace_bytes(32, 32, 32, lbgb.LB_FP32 | lbgb.LB_ONE_COMPONENT, 0)
    two = lbgb.lb_workspace_bytes(32, 32, 32, lbgb.LB_FP32, 0)
    assert 2 * 19 * 4 * N < one < 2 * 19 * 4 * N + (1 << 20) and one < two / 2
    with pytest.raises(lbgb.LBError):
        lbgb.lb_workspace_bytes(32, 32, 32, lbgb.LB_FP32 | lbgb.LB_ONE_COMPONENT, 1)


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle, and LBLattice refuses to run
    without a GPU."""
    pkg = os.path.join(ROOT, "paper_2004_04080_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), f
    import torch

    if not torch.cuda.is_available():
        from paper_2004_04080_gb300.lbgb import LBLattice

        with pytest.raises(RuntimeError):
            LBLattice((8, 8, 8))
