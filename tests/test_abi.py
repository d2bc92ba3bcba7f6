"""The C ABI library builds for sm_103a, loads, and exports every entry point its header declares.

No compute calls here (no GPU in this environment): only the boundary itself."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1308_4908_gb300 import build, hdr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdr_lpa.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(hdr_[a-z_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hdr_create", "hdr_destroy", "hdr_set_rig", "hdr_reconstruct", "hdr_reconstruct_host",
              "hdr_check", "hdr_last_error", "hdr_params_default", "hdr_reconstruct_levels",
              "hdr_reconstruct_batch", "hdr_tune_batch", "hdr_server_create", "hdr_submit", "hdr_poll",
              "hdr_server_stats_get", "hdr_server_destroy", "hdr_calpa_gradients", "hdr_calpa_metric",
              "hdr_reconstruct_steered", "hdr_reconstruct_adaptive"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_c_names(lib):
    for n in declared_functions():
        assert hasattr(hdr, n), n


STRUCTS = ("hdr_sensor_desc", "hdr_params", "hdr_frame", "hdr_batch_config", "hdr_server_config", "hdr_request",
           "hdr_result", "hdr_server_stats", "hdr_calpa_params")


def test_struct_layout_matches_the_header(tmp_path):
    """Every ctypes mirror agrees with the C compiler's layout: size and the offset of every field."""
    lines, want = [], []
    for name in STRUCTS:
        cls = getattr(hdr, name)
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        want.append(ctypes.sizeof(cls))
        for field, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {field}));')
            want.append(getattr(cls, field).offset)
    src = tmp_path / "probe.c"
    src.write_text(f'''#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
{chr(10).join(lines)}
  return 0;
}}''')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    assert got == want


def test_defaults_without_a_gpu(lib):
    p = hdr.hdr_params_default()
    assert p.order == 2 and p.n_scales == 4
    assert [p.sigma[i] for i in range(4)] == [0.5, 0.8, 1.2, 1.8]
    assert abs(p.green_ratio - 2 ** -0.5) < 1e-15 and p.trunc_k == 3.0 and p.ici_gamma == 2.0
    assert p.min_pivot == 1e-3 and p.cond_fallback == 1e6
    c = hdr.hdr_calpa_params_default()
    assert (c.grad_sigma, c.window_sigma, c.alpha, c.lambda1, c.lambda2, c.min_eig, c.max_eig, c.grad_scale) == \
        (1.2, 1.0, 0.3, 1.0, 1e-3, 0.25, 16.0, 0.1)


def test_create_fails_loudly_without_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hdr.HdrError):
        hdr.hdr_create(0)
    with pytest.raises(RuntimeError):
        hdr.Context(0)
