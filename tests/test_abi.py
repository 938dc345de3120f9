"""The C-ABI library loads and exports every function include/eventtracer.h
declares (no compute calls: this runs without a GPU)."""
import os
import re


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(et_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["et_build_scene", "et_render_frames", "et_threshold_events", "et_evsnet_forward",
              "et_scene_free", "et_status_str"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2508_18071_gb300 import _lib
    lib = _lib.load()
    for n in sorted(_declared()):
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n
    assert lib.et_status_str(_lib.ET_ERR_ARG) == b"invalid argument"


def test_oracle_is_not_linked_by_the_library():
    from paper_2508_18071_gb300 import _lib
    import subprocess
    path = _lib.load()._name
    out = subprocess.run(["ldd", path], capture_output=True, text=True).stdout
    assert "oracle" not in out
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2508_18071_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def _prototypes():
    """name -> number of parameters of every et_ function include/eventtracer.h declares."""
    out = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(et_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", src):
            params = m.group(2).strip()
            out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_ctypes_signatures_match_the_header():
    from paper_2508_18071_gb300 import _lib
    protos = _prototypes()
    assert set(protos) == _declared()
    for name, n in protos.items():
        assert len(_lib.SIGNATURES[name][1]) == n, (name, n, _lib.SIGNATURES[name][1])


def test_ctypes_structures_match_the_c_layout(tmp_path):
    """Every structure the binding passes by pointer has the C compiler's size
    and field offsets (compiled from the header with gcc)."""
    import ctypes
    import shutil
    import subprocess
    import pytest
    from paper_2508_18071_gb300 import _lib
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = [_lib.et_material, _lib.et_quad_light, _lib.et_camera, _lib.et_sensor_params,
               _lib.et_evsnet_weights, _lib.et_evsnet_state, _lib.et_train_shape]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "eventtracer.h"', "int main(void) {"]
    for s in structs:
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (s.__name__, s.__name__))
        for f, _ in s._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s.__name__, f, s.__name__, f))
    lines.append('  printf("et_event %zu\\n", sizeof(et_event));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines))
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for s in structs:
        assert int(got[s.__name__]) == ctypes.sizeof(s), s.__name__
        for f, _ in s._fields_:
            assert int(got["%s.%s" % (s.__name__, f)]) == getattr(s, f).offset, (s.__name__, f)
    assert int(got["et_event"]) == _lib.EVENT_BYTES
