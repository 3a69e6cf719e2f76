"""The C-ABI library loads, exports every call include/dartray.h declares, and
rejects bad grid descriptions on the host before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1709_03802_gb300 as pkg
import synth
from paper_1709_03802_gb300 import dartray as dr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_calls():
    with open(os.path.join(ROOT, "include", "dartray.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dartray_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_call():
    lib = pkg.load()
    names = declared_calls()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pkg.EXPORTED)


def test_params_default():
    p = pkg.dartray_params_default()
    assert p.a_rt == 0.05 and p.n_rays_min == 5 and p.n_rays_max == 40 and p.k0 == 2
    assert p.n_fwhm == 5 and p.k_sca_cap == 3 and p.merge == 1 and p.src_stride == 1


def _desc(grid, **over):
    keep = dict(fc=np.ascontiguousarray(grid.first_child, np.int32),
                lon=np.ascontiguousarray(grid.leaf_of_node, np.int32),
                kr=np.ascontiguousarray(grid.kappa_rho, np.float32),
                em=np.ascontiguousarray(grid.emissivity, np.float32),
                al=np.ascontiguousarray(grid.albedo, np.float32), g=np.ascontiguousarray(grid.g, np.float32))
    keep.update(over)
    d = dr.dartray_grid_desc()
    d.nroot[:] = grid.nroot
    d.root_lo[:] = grid.root_lo
    d.root_size = grid.root_size
    d.n_nodes = keep["fc"].shape[0]
    d.n_leaf = grid.n_leaf
    d.n_lambda = grid.n_lambda
    d.first_child = keep["fc"].ctypes.data
    d.leaf_of_node = keep["lon"].ctypes.data
    d.kappa_rho = keep["kr"].ctypes.data
    d.emissivity = keep["em"].ctypes.data
    d.albedo = keep["al"].ctypes.data
    d.g = keep["g"].ctypes.data
    return d, keep


def _create(d):
    lib = pkg.load()
    h = C.c_void_p()
    rc = lib.dartray_grid_create(C.byref(d), None, None, C.byref(h))
    return rc, lib.dartray_last_error().decode()


def test_rejects_cyclic_tree():
    grid = synth.config1(as_tree=True)
    fc = np.ascontiguousarray(grid.first_child, np.int32).copy()
    fc[9] = 1  # a child pointing back into the tree
    d, keep = _desc(grid, fc=fc)
    rc, msg = _create(d)
    assert rc == -1 and msg


def test_rejects_bad_leaf_ids():
    grid = synth.config1()
    lon = np.ascontiguousarray(grid.leaf_of_node, np.int32).copy()
    lon[5] = lon[6]
    d, keep = _desc(grid, lon=lon)
    rc, msg = _create(d)
    assert rc == -1 and "leaf" in msg


def test_rejects_inexact_coordinates():
    grid = synth.config1()
    d, keep = _desc(grid)
    d.root_size = 2.0 / 9.0
    rc, msg = _create(d)
    assert rc == -1 and "exact" in msg


def test_rejects_bad_albedo():
    grid = synth.config1()
    d, keep = _desc(grid, al=np.array([1.5], np.float32))
    rc, msg = _create(d)
    assert rc == -1


@pytest.mark.parametrize("n", [0, 17])
def test_rejects_unsupported_lambda_count(n):
    """1 to 16 wavelengths (counts between the marcher widths 1, 2, 4, 8, 16
    are padded inside the library)."""
    grid = synth.config1()
    d, keep = _desc(grid)
    d.n_lambda = n
    rc, msg = _create(d)
    assert rc == -1 and "n_lambda" in msg


@pytest.mark.parametrize("case", ["deterministic", "nine_wavelengths"])
def test_forward_mode_rejections(case):
    """The forward mode (tangent_albedo) takes at most 8 wavelengths and no
    deterministic mode; both are refused before any device work."""
    grid = synth.config1()
    d, keep = _desc(grid)
    p = dr.dartray_params()
    dr.load().dartray_params_default(C.byref(p))
    p.tangent_albedo = 1
    if case == "deterministic":
        p.deterministic = 1
    else:
        d.n_lambda = 9
    h = C.c_void_p()
    rc = dr.load().dartray_grid_create(C.byref(d), C.byref(p), None, C.byref(h))
    assert rc == -1 and "forward mode" in dr.load().dartray_last_error().decode()


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program built with
    the system compiler against include/dartray.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = [f'printf("%zu\\n", sizeof({struct}));']
    lines += [f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"dartray.h\"\n"
                   "int main(void) {\n" + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("cls", [dr.dartray_grid_desc, dr.dartray_params, dr.dartray_stats, dr.dartray_dust],
                         ids=lambda c: c.__name__)
def test_binding_structs_match_the_header_layout(cls, tmp_path):
    """The ctypes mirrors of the ABI structs have the header's size and the
    same offset for every field."""
    fields = [name for name, _ in cls._fields_]
    size, offsets = _c_layout(cls.__name__, fields, tmp_path)
    assert C.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offsets


def test_octant_mode_rejects_an_asymmetric_model():
    """The octant mode needs a model symmetric about its centre: config 1's
    source sits off the centre, so the grid is refused before any device
    work."""
    grid = synth.config1()
    d, keep = _desc(grid)
    p = pkg.dartray_params_default()
    p.octant = 1
    lib = pkg.load()
    h = C.c_void_p()
    rc = lib.dartray_grid_create(C.byref(d), C.byref(p), None, C.byref(h))
    assert rc == -1 and "octant" in lib.dartray_last_error().decode()
