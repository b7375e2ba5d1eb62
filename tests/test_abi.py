"""CPU checks of the boundary: the C-ABI library builds, loads and exports every
symbol include/dppt.h declares; the ctypes structures match the header's layout; every
entry point turns null arguments and bad devices into status codes.  No compute call is
made (there may be no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "dppt.h")).read()
    return sorted(set(re.findall(r"\b(dppt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2607_13265_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2607_13265_gb300 import _lib
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(_lib.SIGNATURES), "binding and header disagree"


def test_version_string(lib):
    assert lib.dppt_version().decode().startswith("dppt")


def test_struct_layouts_match_header():
    """Sizes of the ctypes mirrors equal the C structs (checked with a tiny C program)."""
    from paper_2607_13265_gb300 import _lib
    import subprocess
    import tempfile
    src = r'''
#include <stdio.h>
#include "dppt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(dppt_material), sizeof(dppt_scene_desc), sizeof(dppt_job),
         sizeof(dppt_params), sizeof(dppt_grads), sizeof(dppt_launch), sizeof(dppt_replay));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    mine = [ctypes.sizeof(t) for t in (_lib.Material, _lib.SceneDesc, _lib.Job, _lib.Params, _lib.Grads, _lib.Launch,
                                      _lib.Replay)]
    assert sizes == mine


def test_field_offsets_match_header():
    """Every field of every ctypes mirror sits at the offset the C compiler gives the
    field of the same name (the Python name `pass_` mirrors the C field `pass`)."""
    from paper_2607_13265_gb300 import _lib
    import subprocess
    import tempfile
    mirrors = {"dppt_material": _lib.Material, "dppt_scene_desc": _lib.SceneDesc, "dppt_job": _lib.Job,
               "dppt_params": _lib.Params, "dppt_grads": _lib.Grads, "dppt_launch": _lib.Launch,
               "dppt_replay": _lib.Replay}
    lines, expect = [], []
    for cname, t in mirrors.items():
        for f in t._fields_:
            name = f[0]
            cfield = "pass" if name == "pass_" else name
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {cfield}));')
            expect.append(getattr(t, name).offset)
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"dppt.h\"\nint main(void) {\n" + "\n".join(lines) + \
          "\n  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "o.c")
        exe = os.path.join(d, "o")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    assert got == expect


def test_missing_library_fails_loudly(tmp_path):
    from paper_2607_13265_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(_lib.DpptError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_null_arguments_return_status_codes(lib):
    """Host-side fault handling: every entry point called with a null context and null or zero
    arguments returns DPPT_ERR_INVALID_ARG (the void ones return), touching no device."""
    from paper_2607_13265_gb300 import _lib
    ints = (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t)
    for name, (res, args) in sorted(_lib.SIGNATURES.items()):
        vals = [0 if a in ints else 0.0 if a in (ctypes.c_float, ctypes.c_double) else None for a in args]
        r = getattr(lib, name)(*vals)
        if name == "dppt_version":
            continue
        if name == "dppt_last_error":
            assert r.decode() == "null context"
        elif res is None:
            assert r is None, name
        else:
            assert r == -1, (name, r)               # DPPT_ERR_INVALID_ARG


def test_create_rejects_bad_devices(lib):
    import torch
    ctx = ctypes.c_void_p()
    for dev in (-1, 1 << 20):
        assert lib.dppt_create(ctypes.byref(ctx), dev) == -1 and not ctx.value
    if not torch.cuda.is_available():            # no device at all: a status code, not a crash
        assert lib.dppt_create(ctypes.byref(ctx), 0) == -1 and not ctx.value
