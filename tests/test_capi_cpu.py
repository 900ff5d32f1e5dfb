"""Boundary checks that need no GPU: the library builds, loads, exports every symbol that
``include/ptycho.h`` declares, and rejects bad arguments on the host before any launch."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptycho.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2311_14780_gb300 import _native, build
    if not os.path.exists(build.lib_path()):
        build.build()
    return _native.lib()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ptycho_[a-z_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_symbols()
    for must in ("ptycho_plan_create", "ptycho_plan_destroy", "ptycho_forward", "ptycho_loss",
                 "ptycho_adjoint", "ptycho_step", "ptycho_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(lib._name)
    for name in declared_symbols():
        assert hasattr(raw, name), name


def test_binding_declares_every_exported_symbol():
    from paper_2311_14780_gb300 import _native
    bound = {s[0] for s in _native.SIGNATURES}
    assert set(declared_symbols()) <= bound | {"ptycho_plan_create"}


def test_python_flag_constants_match_the_header():
    from paper_2311_14780_gb300 import api
    text = open(HEADER).read()
    flags = dict((k, int(v)) for k, v in re.findall(r"#define PTYCHO_FLAG_([A-Z0-9_]+) (\d+)", text))
    assert flags
    for name, value in flags.items():
        assert getattr(api, "FLAG_" + name) == value, name
    assert len(set(flags.values())) == len(flags)                          # distinct bits
    assert all(v & (v - 1) == 0 for v in flags.values())


def test_strerror(lib):
    assert lib.ptycho_strerror(0) == b"success"
    assert b"outside" in lib.ptycho_strerror(-2)
    assert lib.ptycho_strerror(-99) == b"unknown error"


def _geom(F=64, L=1, M=1, J=2, H=80, W=80, pos=None, loss=0, remap=0, tilt=1.2):
    from paper_2311_14780_gb300 import _native
    g = _native.Geom()
    keep = {}
    keep["h"] = np.full(L, H, np.int32)
    keep["w"] = np.full(L, W, np.int32)
    keep["pos"] = np.zeros((L, J, 2), np.int32) if pos is None else np.ascontiguousarray(pos, np.int32)
    g.L, g.M, g.F, g.J = L, M, F, J
    g.obj_h = keep["h"].ctypes.data_as(_native.c_int32_p)
    g.obj_w = keep["w"].ctypes.data_as(_native.c_int32_p)
    g.pos = keep["pos"].ctypes.data_as(_native.c_int32_p)
    g.z, g.det_pixel, g.tilt_rad = 0.088, 15e-6, tilt
    g.remap, g.loss, g.eps = remap, loss, 0.0
    return g, keep


@pytest.mark.parametrize("kw,code", [
    (dict(F=100), -6),            # frame size not supported
    (dict(L=17, J=1), -6),        # more wavelengths than the ABI supports
    (dict(L=0), -1),
    (dict(M=0), -1),
    (dict(J=0), -1),
    (dict(loss=7), -1),
    (dict(H=32), -1),             # object smaller than a frame
    (dict(remap=1, tilt=2.0), -1),
])
def test_plan_create_rejects_bad_geometry_on_the_host(lib, kw, code):
    g, keep = _geom(**kw)
    h = ctypes.c_void_p()
    assert lib.ptycho_plan_create(ctypes.byref(g), ctypes.byref(h)) == code
    assert not h.value


@pytest.mark.parametrize("bad", [(17, 0), (0, 17), (-1, 0), (0, -1)])
def test_plan_create_rejects_patches_outside_the_object(lib, bad):
    pos = np.zeros((1, 2, 2), np.int32)
    pos[0, 1] = bad
    g, keep = _geom(pos=pos)
    h = ctypes.c_void_p()
    assert lib.ptycho_plan_create(ctypes.byref(g), ctypes.byref(h)) == -2


def test_null_arguments_are_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.ptycho_plan_create(None, ctypes.byref(h)) == -1
    assert lib.ptycho_forward(None, None, None, None, None, None, None) == -1
    assert lib.ptycho_plan_destroy(None) == 0


def test_tilt_correct_rejects_bad_arguments_on_the_host(lib):
    """Argument errors are caught before any CUDA call (so this runs without a GPU)."""
    f = lib.ptycho_tilt_correct
    a, b = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x100000)
    ok = dict(F=64, J=3, z=0.02, p=15e-6, t=1.2, lo=-math.inf, hi=math.inf)

    def call(**kw):
        k = {**ok, **kw}
        return f(k["F"], k["J"], k["z"], k["p"], k["t"], kw.get("cam", a), k["lo"], k["hi"], kw.get("out", b),
                 None, None)

    assert call(F=1) == -1 and call(F=9000) == -1 and call(J=-1) == -1
    assert call(z=0.0) == -1 and call(p=-1e-6) == -1 and call(z=math.inf) == -1
    assert call(t=math.pi / 2) == -1 and call(t=math.nan) == -1
    assert call(lo=5.0, hi=5.0) == -1 and call(lo=math.nan) == -1 and call(hi=math.nan) == -1
    assert call(cam=None) == -1 and call(out=None) == -1
    assert call(out=ctypes.c_void_p(0x1000 + 64 * 64 * 4)) == -1          # output overlaps the input
    assert call(J=0, cam=None, out=None) == 0                            # nothing to do, nothing launched
    # the table / apply split
    assert lib.ptycho_tilt_table_bytes(256) == 256 * 256 * 20 and lib.ptycho_tilt_table_bytes(1) == -1
    assert lib.ptycho_tilt_table_bytes(101) == 101 * 101 * 20
    assert lib.ptycho_tilt_table(64, 0.02, 15e-6, 1.2, None, None) == -1
    assert lib.ptycho_tilt_table(64, 0.02, 15e-6, 1.2, ctypes.c_void_p(0x1008), None) == -1   # misaligned
    assert lib.ptycho_tilt_table(64, -0.02, 15e-6, 1.2, a, None) == -1
    tab = ctypes.c_void_p(0x200000)
    ap = lib.ptycho_tilt_apply
    assert ap(64, 3, None, a, -math.inf, math.inf, b, None, None) == -1
    assert ap(64, 3, ctypes.c_void_p(0x200008), a, -math.inf, math.inf, b, None, None) == -1
    assert ap(64, 3, tab, a, 2.0, 1.0, b, None, None) == -1
    assert ap(64, 3, tab, a, -math.inf, math.inf, ctypes.c_void_p(0x200000 + 64), None, None) == -1  # out on the table
    assert ap(64, 3, tab, a, -math.inf, math.inf, b, ctypes.c_void_p(0x100010), None) == -1        # mask on out
    assert ap(64, 0, None, None, -math.inf, math.inf, None, None, None) == 0


def test_regularise_rejects_bad_arguments_on_the_host(lib):
    f = lib.ptycho_regularise
    a = ctypes.c_void_p(0x1000)
    assert f(None, a, 0.1, 0.1, 1e-3, a, None, None) == -1
    fake_plan = ctypes.c_void_p(0x2000)        # never dereferenced: the checks below come first
    assert f(fake_plan, None, 0.1, 0.1, 1e-3, a, None, None) == -1
    assert f(fake_plan, a, 0.1, 0.1, 1e-3, None, None, None) == -1
    assert f(fake_plan, a, -0.1, 0.1, 1e-3, a, None, None) == -1
    assert f(fake_plan, a, 0.1, 0.1, 0.0, a, None, None) == -1
    assert f(fake_plan, a, math.nan, 0.1, 1e-3, a, None, None) == -1
    assert f(fake_plan, a, 0.1, math.inf, 1e-3, a, None, None) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2311_14780_gb300 import _native
    monkeypatch.setattr(_native, "_LIB", None)
    monkeypatch.setattr(_native, "lib_path", lambda: str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _native.lib()


def test_noalloc_forward_rejects_what_it_cannot_do_before_touching_the_gpu(lib):
    """The allocation-free forward entry point checks every size and position on the host
    before it asks for a device: an unsupported frame size, a problem whose tables alone do
    not fit its fixed array, and a patch outside its object.  The data pointers here are
    placeholders that are never dereferenced."""
    ip = ctypes.POINTER(ctypes.c_int32)
    fake = ctypes.c_void_p(256)

    def call(L, M, F, J, H, pos):
        h = np.full(L, H, np.int32)
        w = np.full(L, H, np.int32)
        pos = np.ascontiguousarray(pos, np.int32)
        return lib.ptycho_forward_noalloc(L, M, F, J, h.ctypes.data_as(ip), w.ctypes.data_as(ip),
                                          pos.ctypes.data_as(ip), fake, fake, None, None, fake, None)

    assert call(1, 1, 100, 4, 128, np.zeros((1, 4, 2))) == -6                 # F not in {64,128,256,512}
    assert call(1, 1, 64, 3_000_000, 128, np.zeros((1, 3_000_000, 2))) == -7  # position tables exceed the array
    assert b"fixed array" in lib.ptycho_strerror(-7)
    bad = np.zeros((2, 4, 2))
    bad[1, 3] = (70, 0)                                                       # 70 + 64 > 128
    assert call(2, 1, 64, 4, 128, bad) == -2
    assert call(1, 1, 64, 0, 128, np.zeros((1, 1, 2))) == -1                  # no positions
