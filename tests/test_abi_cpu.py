"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
entry point include/lpm.h declares, the ctypes record matches the C layout, and invalid
configurations are rejected before any CUDA call."""
import ctypes as C
import dataclasses
import os
import re
import subprocess

import numpy as np
import pytest

import lpm_inputs as li
from paper_0912_3223_gb300 import build as pkg_build
from paper_0912_3223_gb300 import lpm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lpm.h")


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return lpm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lpm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lpm_create", "lpm_set_met", "lpm_release", "lpm_step",
                     "lpm_concentration", "lpm_deposition", "lpm_destroy"):
        assert required in names
    assert sorted(lpm.SYMBOLS) == names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lpm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lpm_[a-z_]+)\b", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_config_layout_matches_c_header(tmp_path):
    fields = [f for f, _ in lpm.lpm_config._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"',
            "int main(void) {", 'printf("%zu\\n", sizeof(lpm_config));']
    prog += [f'printf("%zu\\n", offsetof(lpm_config, {f}));' for f in fields]
    prog += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals[0] == C.sizeof(lpm.lpm_config)
    for f, off in zip(fields, vals[1:]):
        assert getattr(lpm.lpm_config, f).offset == off, f


@pytest.mark.parametrize("mutate,msg", [
    (dict(nx=1), "at least 2 nodes"),
    (dict(dt=0.0), "dt must be"),
    (dict(bin_every=0), "bin_every"),
    (dict(cx=0), "non-empty"),
    (dict(n_steps=0), "n_steps"),
    (dict(nz=65), "exceeds 64 levels"),
    (dict(vd_dry=0.01, h_mix=0.0), "h_mix"),
    (dict(reflect_top=1, z_top=0.0), "z_top"),
    (dict(n_scenarios=0), "n_scenarios"),
])
def test_invalid_configs_rejected_on_host(lib, mutate, msg):
    cfg = dataclasses.replace(li.make_cfg0(n_particles=10, n_steps=10), **mutate)
    with pytest.raises(lpm.LpmError) as e:
        lpm.lpm_create(cfg)
    assert e.value.status == lpm.LPM_E_INVALID
    assert msg in str(e.value)


def test_descending_levels_rejected(lib):
    cfg = li.make_cfg0(n_particles=10, n_steps=10)
    cfg = dataclasses.replace(cfg, z_levels=np.array([0.0, 0.0]))
    with pytest.raises(lpm.LpmError, match="ascending"):
        lpm.lpm_create(cfg)


def test_oracle_and_cuda_path_share_no_code():
    """The oracle neither imports nor includes the product package, and vice versa."""
    for path in ("oracle/__init__.py", "oracle/lpm_oracle.c"):
        text = open(os.path.join(ROOT, path)).read()
        assert "paper_0912_3223_gb300" not in text and "csrc" not in text
    pkg = os.path.join(ROOT, "paper_0912_3223_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lpm_oracle" not in text, f


def test_context_calls_reject_a_null_context(lib):
    """Every context call checks its context before touching the device: NULL gives
    LPM_E_INVALID (here, with no GPU, any CUDA call would fail differently)."""
    vp = C.c_void_p(None)
    i64 = C.c_int64
    calls = [
        lambda: lib.lpm_step(vp, i64(1)),
        lambda: lib.lpm_reset(vp),
        lambda: lib.lpm_sync(vp),
        lambda: lib.lpm_set_sort(vp, 60),
        lambda: lib.lpm_set_launch(vp, 512, 1, 2),
        lambda: lib.lpm_set_params(vp, 1.0, 0.0, 0.0),
        lambda: lib.lpm_set_profiling(vp, 1),
        lambda: lib.lpm_set_dosage(vp, 4),
        lambda: lib.lpm_set_langevin(vp, 1, 100.0),
        lambda: lib.lpm_set_adjoint_storage(vp, 0),
        lambda: lib.lpm_adjoint_storage(vp, C.byref(C.c_int()), C.byref(C.c_uint64())),
        lambda: lib.lpm_concentration(vp, 0, None, 0),
        lambda: lib.lpm_deposition(vp, 0, None, None, 0),
        lambda: lib.lpm_budget(vp, 0, (C.c_double * 8)()),
        lambda: lib.lpm_current_step(vp, C.byref(i64())),
    ]
    for call in calls:
        assert call() == lpm.LPM_E_INVALID


def test_product_path_fails_loudly_without_the_library_or_a_gpu(monkeypatch, tmp_path):
    """No fallback: a missing liblpm.so raises on load, and a simulation without a CUDA
    device raises instead of running anywhere else."""
    import torch
    from paper_0912_3223_gb300 import Sim
    monkeypatch.setattr(lpm, "LIB_PATH", str(tmp_path / "liblpm.so"))
    monkeypatch.setattr(lpm, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        lpm.load()
    if not torch.cuda.is_available():
        with pytest.raises(RuntimeError, match="CUDA GPU"):
            Sim(li.make_cfg0(n_particles=10, n_steps=10))
