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


def test_setup_rejects_bad_batch_width_without_gpu():
    """batch_cols must be 2, 4, 8, 16 or 32: checked with the other parameters, before any device work."""
    import numpy as np

    import paper_2601_04112_gb300 as amg

    lib = amg.load_library()
    rp = np.array([0, 2, 4], dtype=np.int64)
    cl = np.array([0, 1, 1, 2], dtype=np.int32)
    vl = np.ones(4)
    csr = amg.Csr(m=2, n=3, nnz=4, rowptr=rp.ctypes.data, col=cl.ctypes.data, val=vl.ctypes.data, mem=amg.HOST)
    for bad in (0, 3, 12, 64):
        prm = amg.params(batch_cols=bad)
        h = ctypes.c_void_p()
        st = lib.amgdd_setup(ctypes.byref(csr), None, None, 1, ctypes.byref(prm), None, ctypes.byref(h))
        assert st == -1 and b"invalid parameters" in lib.amgdd_last_error(), (bad, st)


def _saved_file(path, n, levels, params_bytes):
    """A saved-hierarchy file of the current format: setup inputs of a path graph on n unknowns (rows {j, j+1}),
    no kernel choices, then the level snapshots given as dicts (missing vectors empty)."""
    import struct

    import numpy as np

    rowptr = np.arange(0, 2 * (n - 1) + 1, 2, dtype=np.int64)
    col = np.array(sum(([j, j + 1] for j in range(n - 1)), []), dtype=np.int32)
    val = np.ones(col.shape[0])
    agg = np.zeros(n, dtype=np.int32)

    def vec(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        return struct.pack("<Q", a.shape[0]) + a.tobytes()

    out = b"AMGDDHv2" + struct.pack("<I", len(params_bytes)) + params_bytes + struct.pack("<iiq", 1, 0, n)
    out += vec(rowptr, np.int64) + vec(col, np.int32) + vec(val, np.float64) + vec(agg, np.int32)
    out += vec([], np.float64) + struct.pack("<Q", 0) + struct.pack("<Q", len(levels))
    for L in levels:
        out += struct.pack("<qqiiiiiidd", L["n"], 0, L.get("nagg", 0), L["coarsest"], 0, 0, 0, 0, 0.1, 0.0)
        for key in ("g_ptr", "h_off", "om_ptr", "z_off", "mu_off", "col0", "wf_off"):
            out += vec(L.get(key, []), np.int64)
        for key in ("g_idx", "g_rank", "agg", "om_idx", "nomega", "k"):
            out += vec(L.get(key, []), np.int32)
        for key in ("R64", "W64", "Aw64", "mu", "Z64", "Wf64", "A64"):
            out += vec(L.get(key, []), np.float64)
    path.write_bytes(out)


def test_hierarchy_load_checks_every_level_before_device_work(tmp_path):
    """A file whose level snapshots disagree with themselves is refused on the host (AMGDD_ERR_INVALID_ARG),
    before any index of it reaches the device: a stored matrix of the wrong size, compressed rows that do not
    fill their groups, a level that does not end the hierarchy as its coarsest, an Omega list pointing outside
    its level, an aggregate id out of range."""
    import numpy as np

    import paper_2601_04112_gb300 as amg

    lib = amg.load_library()
    prm = amg.params()
    pbytes = ctypes.string_at(ctypes.addressof(prm), ctypes.sizeof(prm))
    n = 4
    g_ptr = np.arange(0, 2 * (n - 1) + 1, 2)
    g_idx = np.array(sum(([j, j + 1] for j in range(n - 1)), []))
    h_off = np.arange(0, 4 * (n - 1) + 1, 4)
    one_level = dict(n=n, coarsest=1, g_ptr=g_ptr, g_idx=g_idx, h_off=h_off, g_rank=[2] * (n - 1),
                     R64=np.ones(4 * (n - 1)), W64=np.eye(n).ravel())
    two = dict(n=n, coarsest=0, nagg=2, g_ptr=g_ptr, g_idx=g_idx, h_off=h_off, g_rank=[2] * (n - 1),
               R64=np.ones(4 * (n - 1)), agg=[0, 0, 1, 1], om_ptr=[0, 3, 6], om_idx=[0, 1, 2, 2, 3, 1],
               nomega=[2, 2], k=[1, 1], col0=[0, 1, 2], z_off=[0, 2, 4], mu_off=[0, 2, 4],
               W64=np.ones(12), mu=np.zeros(4), Z64=np.ones(4))
    coarse = dict(n=2, coarsest=1, g_ptr=[0, 2], g_idx=[0, 1], h_off=[0, 4], W64=np.eye(2).ravel())
    cases = {
        "W of the wrong size": [dict(one_level, W64=np.ones(n * n - 1))],
        "rows short of their groups": [dict(one_level, R64=np.ones(4 * (n - 1) - 2))],
        "a rank above its support": [dict(one_level, g_rank=[3] * (n - 1))],
        "no coarsest level at the end": [dict(one_level, coarsest=0)],
        "Omega outside the level": [dict(two, om_idx=[0, 1, 2, 2, 3, 9]), coarse],
        "aggregate id out of range": [dict(two, agg=[0, 0, 1, 2]), coarse],
        "next level of the wrong size": [two, dict(coarse, n=3, W64=np.eye(3).ravel())],
        "k above its omega": [dict(two, k=[3, 1], col0=[0, 3, 4], z_off=[0, 6, 8], Z64=np.ones(8)), coarse],
    }
    for name, levels in cases.items():
        path = tmp_path / "h.amgdd"
        _saved_file(path, n, levels, pbytes)
        h = ctypes.c_void_p()
        st = lib.amgdd_hierarchy_load(str(path).encode(), None, ctypes.byref(h))
        assert st == -1, (name, st, lib.amgdd_last_error())
        assert b"not a saved hierarchy" in lib.amgdd_last_error(), name
    # controls: the same files made consistent pass the host checks (without a GPU they then stop at the device)
    for levels in ([one_level], [two, coarse]):
        path = tmp_path / "ok.amgdd"
        _saved_file(path, n, levels, pbytes)
        h = ctypes.c_void_p()
        st = lib.amgdd_hierarchy_load(str(path).encode(), None, ctypes.byref(h))
        if st == 0:
            lib.amgdd_free(h)
        else:
            assert b"not a saved hierarchy" not in lib.amgdd_last_error(), lib.amgdd_last_error()
