"""The C ABI without a GPU: the library loads, exports every symbol that
include/freeray.h declares, and the ctypes mirrors of its structures have the
layout a C compiler gives them."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "freeray.h")


@pytest.fixture(scope="module")
def freeray():
    from paper_2302_12031_gb300 import _build, api
    _build.build()
    return api


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_path():
    names = declared_functions()
    for need in ("fr_trace_forward", "fr_trace_adjoint", "fr_loss_l2", "fr_adam_step", "fr_trace_debug",
                 "fr_trace_batch_forward", "fr_trace_batch_adjoint", "fr_create", "fr_destroy", "fr_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(freeray):
    lib = C.CDLL(freeray.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(freeray._SIGNATURES)


def test_abi_version_without_gpu(freeray):
    assert freeray.fr_abi_version() == freeray.ABI_VERSION == 3


def test_null_handle_is_an_argument_error(freeray):
    L = freeray.lib()
    assert L.fr_destroy(None) == 0
    assert L.fr_trace_forward(None, None, None, None, 1, 0, 0, 1, None, None, None, None) == 1
    assert L.fr_stream_wait(None, None, 1) == 1
    assert L.fr_last_error(None) == b"null handle"


def test_struct_layouts_match_the_c_compiler(tmp_path, freeray):
    structs = {"fr_lens_desc": freeray.LensDesc, "fr_source_desc": freeray.SourceDesc,
               "fr_target_desc": freeray.TargetDesc, "fr_options": freeray.Options,
               "fr_stats": freeray.Stats, "fr_ray_record": freeray.RayRecord,
               "fr_batch_item": freeray.BatchItem}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "freeray.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(out[cname]) == C.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert int(out["%s.%s" % (cname, field)]) == getattr(cls, field).offset, (cname, field)


def test_options_marshalling_without_gpu(freeray):
    import torch
    o = freeray.make_options(hist_mode=3, window_cells=1234, mesh=(2, 3))
    assert (o.hist_mode, o.window_cells, o.mesh_nu, o.mesh_nv) == (3, 1234, 2, 3)
    assert not o.ray_order and not freeray.BatchItem().ray_order        # NULL: ray-id order
    with pytest.raises(ValueError):
        freeray.make_options(ray_order=torch.zeros(9, dtype=torch.int32))        # host memory
    with pytest.raises(ValueError):
        freeray.make_options(ray_order=torch.zeros(9, dtype=torch.int64))        # not 32-bit ids


def test_ray_order_length_is_checked_against_the_problem(freeray):
    import types
    pb = types.SimpleNamespace(n_rays=10)
    o = freeray.make_options()
    freeray.Problem.check_options(pb, o)                  # no order: nothing to check
    o.ray_order = 0x1000                                  # an address set without its length
    with pytest.raises(ValueError):
        freeray.Problem.check_options(pb, o)
    o.ray_order_numel = 9                                 # built for 8 rays
    with pytest.raises(ValueError):
        freeray.Problem.check_options(pb, o)
    o.ray_order_numel = 11                                # n_rays + 1
    freeray.Problem.check_options(pb, o)
