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
