"""The C-ABI library builds for sm_103a and exports every symbol that
include/amgdd.h declares; its host-only logic (defaults, file checks) runs
here too.  No device call: this runs without a GPU."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(amgdd_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_declared_symbols():
    from paper_2601_04112_gb300 import build

    lib = ctypes.CDLL(build.build())
    names = _declared()
    assert len(names) >= 12
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_lists_every_symbol():
    import paper_2601_04112_gb300 as amg

    assert set(amg.EXPORTED) <= _declared()


def test_params_default_without_gpu():
    import paper_2601_04112_gb300 as amg

    amg.load_library()
    p = amg.params(c_min=(2, 3, 4))
    assert p.L_max == 10 and p.n_coarse == 2000 and abs(p.thresh - 0.1) < 1e-15
    assert list(p.c_min)[:3] == [2, 3, 4] and p.n_cmin == 3
    assert p.kappa == 0.0 and p.agg_passes == 1 and p.batch_cols == 8



def test_hierarchy_load_rejects_bad_files(tmp_path):
    """amgdd_hierarchy_load checks the file before any device work."""
    import paper_2601_04112_gb300 as amg

    amg.load_library()
    bad = tmp_path / "bad.amgdd"
    bad.write_bytes(b"not a hierarchy" * 10)
    for path in (bad, tmp_path / "missing.amgdd"):
        try:
            amg.Hierarchy.load(path)
        except amg.AmgddError as e:
            assert e.status == -1
        else:
            raise AssertionError("load accepted " + str(path))
