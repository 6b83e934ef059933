"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol
``include/tmm.h`` declares, its structs match the header's layout, and the
host-side argument checks reject bad problems before touching a device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_13667_gb300 import build
    build.build()
    from paper_2111_13667_gb300 import abi
    return abi.load()


def declared_symbols():
    out = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            out += re.findall(r"TMM_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)
    return out


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "tmm_coh_batched" in syms and "tmm_coh_grad" in syms
    for s in syms:
        assert hasattr(lib, s), s
    nm = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2111_13667_gb300", "libtmm.so")],
                        capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (tmm_\w+)", nm))
    assert set(syms) <= exported
    from paper_2111_13667_gb300 import abi
    assert set(abi.EXPORTED) <= set(syms)


def test_struct_layout_matches_header(tmp_path, lib):
    from paper_2111_13667_gb300.abi import TmmAdamCfg, TmmLaunchCfg, TmmProblem
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "tmm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(tmm_problem), offsetof(tmm_problem, n_direct),
         offsetof(tmm_problem, mat_table), offsetof(tmm_problem, n_materials), offsetof(tmm_problem, d),
         offsetof(tmm_problem, lambda), sizeof(tmm_launch_cfg), offsetof(tmm_launch_cfg, max_items_per_block));
  printf("%zu %zu %zu\\n", sizeof(tmm_adam_cfg), offsetof(tmm_adam_cfg, d_max), offsetof(tmm_adam_cfg, step0));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(TmmProblem), TmmProblem.n_direct.offset, TmmProblem.mat_table.offset,
            TmmProblem.n_materials.offset, TmmProblem.d.offset, TmmProblem.lambda_.offset,
            ctypes.sizeof(TmmLaunchCfg), TmmLaunchCfg.max_items_per_block.offset,
            ctypes.sizeof(TmmAdamCfg), TmmAdamCfg.d_max.offset, TmmAdamCfg.step0.offset]
    assert got == want


def _problem(**kw):
    from paper_2111_13667_gb300.abi import TmmProblem
    p = TmmProblem()
    p.S, p.L_max, p.n_lambda, p.n_theta, p.pol_mask, p.prec = 4, 3, 8, 2, 3, 0
    p.n_direct = 0x1000
    p.d, p.theta, p.lambda_ = 0x2000, 0x3000, 0x4000
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [
    dict(S=-1), dict(L_max=-2), dict(n_lambda=-1), dict(pol_mask=0), dict(pol_mask=4), dict(pol_mask=5),
    dict(pol_mask=6), dict(pol_mask=8), dict(prec=7),
    dict(mat_table=0x5000),                       # both index sources
    dict(n_direct=None),                          # neither index source
    dict(n_direct_per_lambda=2),
    dict(theta=None), dict(d=None),
    dict(n_direct=None, mat_table=0x5000, mat_idx=0x6000, n_materials=0),
])
def test_host_rejects_bad_problem(lib, bad):
    from paper_2111_13667_gb300 import abi
    p = _problem(**bad)
    st = lib.tmm_coh_batched(ctypes.byref(p), ctypes.c_void_p(0x7000), None, None)
    assert st == abi.TMM_ERR_INVALID_ARG
    n = ctypes.c_size_t(0)
    assert lib.tmm_workspace_size(ctypes.byref(p), None, ctypes.byref(n)) == abi.TMM_ERR_INVALID_ARG


def test_host_rejects_missing_outputs_and_bad_cfg(lib):
    from paper_2111_13667_gb300 import abi
    p = _problem()
    assert lib.tmm_coh_batched(ctypes.byref(p), None, None, None) == abi.TMM_ERR_INVALID_ARG
    cfg = abi.launch_cfg(tile_lambda=-4)
    assert lib.tmm_coh_batched_ex(ctypes.byref(p), ctypes.byref(cfg), None, 0, ctypes.c_void_p(0x7000),
                                  None, None) == abi.TMM_ERR_INVALID_ARG
    cfg = abi.launch_cfg(persistent=2)
    assert lib.tmm_coh_batched_ex(ctypes.byref(p), ctypes.byref(cfg), None, 0, ctypes.c_void_p(0x7000),
                                  None, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_coh_grad(ctypes.byref(p), None, None, None, None, None, 0, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_workspace_status(None, None) == abi.TMM_ERR_INVALID_ARG


def test_optimiser_and_average_mode_argument_checks(lib):
    from paper_2111_13667_gb300 import abi
    fake = ctypes.c_void_p(0x7000)
    p = _problem()
    bad = [abi.adam_cfg(0.0), abi.adam_cfg(1.0, beta1=1.0), abi.adam_cfg(1.0, beta2=-0.1),
           abi.adam_cfg(1.0, eps=0.0), abi.adam_cfg(1.0, d_min=2.0, d_max=1.0), abi.adam_cfg(1.0, step0=-1)]
    for cfg in bad:
        assert lib.tmm_optimize_adam(ctypes.byref(p), fake, ctypes.byref(cfg), 1, None, fake, 1 << 20,
                                     None) == abi.TMM_ERR_INVALID_ARG
    cfg = abi.adam_cfg(1.0)
    assert lib.tmm_optimize_adam(ctypes.byref(p), fake, None, 1, None, fake, 1 << 20, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_optimize_adam(ctypes.byref(p), fake, ctypes.byref(cfg), -1, None, fake, 1 << 20,
                                 None) == abi.TMM_ERR_INVALID_ARG
    px = _problem(prec=abi.TMM_F64X)
    assert lib.tmm_optimize_adam(ctypes.byref(px), fake, ctypes.byref(cfg), 1, None, fake, 1 << 20,
                                 None) == abi.TMM_ERR_UNSUPPORTED
    # the s/p average (pol_mask 7) is a forward output mode; merit and gradients refuse it
    pa = _problem(pol_mask=7)
    assert lib.tmm_coh_grad(ctypes.byref(pa), fake, fake, fake, None, None, 0, None) == abi.TMM_ERR_UNSUPPORTED
    assert lib.tmm_optimize_adam(ctypes.byref(pa), fake, ctypes.byref(cfg), 1, None, fake, 1 << 20,
                                 None) == abi.TMM_ERR_UNSUPPORTED
    n = ctypes.c_size_t(0)
    assert lib.tmm_workspace_size(ctypes.byref(pa), None, ctypes.byref(n)) == abi.TMM_OK


def test_incoherent_absorption_reward_argument_checks(lib):
    from paper_2111_13667_gb300 import abi
    fake = ctypes.c_void_p(0x7000)
    p = _problem()
    px = _problem(prec=abi.TMM_F64X)
    # missing outputs
    assert lib.tmm_inc_batched(ctypes.byref(p), None, None, None, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_absorption_batched(ctypes.byref(p), None, None, None, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_absorption_batched(ctypes.byref(p), fake, None, fake, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_coh_reward(ctypes.byref(p), None, None, fake, fake, 1 << 20, None) == abi.TMM_ERR_INVALID_ARG
    # double-float is the forward kernel's mode only
    assert lib.tmm_inc_batched(ctypes.byref(px), None, fake, None, None) == abi.TMM_ERR_UNSUPPORTED
    assert lib.tmm_absorption_batched(ctypes.byref(px), fake, None, None, None) == abi.TMM_ERR_UNSUPPORTED
    assert lib.tmm_coh_reward(ctypes.byref(px), None, fake, fake, fake, 1 << 20, None) == abi.TMM_ERR_UNSUPPORTED
    # absorption keeps per-layer records: L_max <= 127
    big = _problem(L_max=200)
    assert lib.tmm_absorption_batched(ctypes.byref(big), fake, None, None, None) == abi.TMM_ERR_UNSUPPORTED
    # partial coherence: node count, pointers, precision
    lay = ctypes.c_void_p(0x7100)
    assert lib.tmm_pcoh_batched(ctypes.byref(p), lay, fake, 0, fake, None, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_pcoh_batched(ctypes.byref(p), lay, fake, 257, fake, None, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_pcoh_batched(ctypes.byref(p), None, fake, 8, fake, None, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_pcoh_batched(ctypes.byref(p), lay, None, 8, fake, None, None) == abi.TMM_ERR_INVALID_ARG
    assert lib.tmm_pcoh_batched(ctypes.byref(px), lay, fake, 8, fake, None, None) == abi.TMM_ERR_UNSUPPORTED
    # the field profile only stages the stack in shared memory
    deep = _problem(L_max=100000)
    assert lib.tmm_field_profile(ctypes.byref(deep), 2, fake, None) == abi.TMM_ERR_UNSUPPORTED
    assert lib.tmm_field_profile(ctypes.byref(p), 0, fake, None) == abi.TMM_ERR_INVALID_ARG
    # a reward launch has no status channel for an iteration limit
    cfg = abi.launch_cfg(persistent=1, max_items_per_block=3)
    assert lib.tmm_coh_reward(ctypes.byref(p), ctypes.byref(cfg), fake, fake, fake, 1 << 20,
                              None) == abi.TMM_ERR_INVALID_ARG
    # empty batches are no-ops
    e = _problem(S=0)
    assert lib.tmm_inc_batched(ctypes.byref(e), None, None, None, None) == abi.TMM_OK
    assert lib.tmm_absorption_batched(ctypes.byref(e), None, None, None, None) == abi.TMM_OK
    assert lib.tmm_coh_reward(ctypes.byref(e), None, None, None, None, 0, None) == abi.TMM_OK
    assert lib.tmm_pcoh_batched(ctypes.byref(e), None, None, 8, None, None, None) == abi.TMM_OK


def test_empty_problem_is_a_noop(lib):
    from paper_2111_13667_gb300 import abi
    p = _problem(S=0)
    assert lib.tmm_coh_batched(ctypes.byref(p), None, None, None) == abi.TMM_OK


def test_status_strings(lib):
    from paper_2111_13667_gb300 import abi
    assert lib.tmm_status_string(abi.TMM_OK) == b"ok"
    assert b"argument" in lib.tmm_status_string(abi.TMM_ERR_INVALID_ARG)
    assert lib.tmm_version() >= 100


def test_product_package_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2111_13667_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "tmm_oracle" not in txt, f
