"""Host-only checks of the C ABI (no GPU needed).

- libgs103.so loads and exports every function declared in include/gs.h;
- the ctypes structures match the C layouts field by field (checked against
  offsetof/sizeof printed by a C program compiled from the header);
- argument errors are rejected on the host before anything is enqueued.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2409_18122_gb300 import _lib as L
from paper_2409_18122_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    B.build()
    return L.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gs_status|const char\*|uint64_t)\s+(gs_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10 and "gs_kernel_launches" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.PROTOTYPES, n


def test_struct_layouts_match_header(tmp_path):
    structs = {
        "gs_camera": L.gs_camera, "gs_map": L.gs_map, "gs_params": L.gs_params, "gs_proj": L.gs_proj,
        "gs_bins": L.gs_bins, "gs_image": L.gs_image, "gs_image_grad": L.gs_image_grad, "gs_map_grad": L.gs_map_grad,
        "gs_utility_params": L.gs_utility_params, "gs_region_grid": L.gs_region_grid,
        "gs_loss_weights": L.gs_loss_weights, "gs_adam_params": L.gs_adam_params,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', "int main(void) {"]
    for s, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for s, cls in structs.items():
        assert int(out[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(out["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)


def test_status_strings_and_version(lib):
    assert lib.gs_version().decode().count(".") == 2
    for code in range(7):
        assert lib.gs_status_str(code).decode().startswith("GS_")


def test_workspace_sizes(lib):
    # binning scratch grows with the record and tile capacities; pairs are written straight to gs_bins
    a = L.workspace_size(L.GS_OP_BIN_SORT, 1000, 2, 2000, 10_000, 100)
    b = L.workspace_size(L.GS_OP_BIN_SORT, 1000, 2, 4000, 10_000, 100)
    assert 0 < a < b and a % 256 == 0
    # with room for many pairs the chunk count is set by the chunk target, and the
    # per-(tile, chunk) count table grows with the tiles
    big = 100_000_000
    assert L.workspace_size(L.GS_OP_BIN_SORT, 1000, 2, 2000, big, 200) > \
        L.workspace_size(L.GS_OP_BIN_SORT, 1000, 2, 2000, big, 100)
    # a larger pair capacity allows more placement chunks (a larger count table), never fewer
    assert L.workspace_size(L.GS_OP_BIN_SORT, 1000, 2, 2000, 20_000, 100) >= a
    assert L.workspace_size(L.GS_OP_RENDER_BWD, 10, 1, 10) >= 48 * 10
    assert L.workspace_size(L.GS_OP_INFO_GAIN, 100, 3, 0, 1000, 64) > 0
    out = ctypes.c_size_t(0)
    assert lib.gs_workspace_size(99, 1, 1, 1, 1, 1, ctypes.byref(out)) == L.GS_ERR_ARG
    assert lib.gs_workspace_size(0, -1, 1, 1, 1, 1, ctypes.byref(out)) == L.GS_ERR_ARG
    assert lib.gs_workspace_size(0, 1, 1, 1, 1, 1, None) == L.GS_ERR_NULL


def _params(**kw):
    d = dict(tile_w=16, tile_h=16, eps2d=0.3, near_plane=0.2, guard=1.3, alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4,
             ig_batch=0, fwd_batch=0)
    d.update(kw)
    return L.gs_params(*d.values())


def test_host_side_argument_errors(lib):
    """Invalid arguments come back as status codes; nothing touches a device."""
    fake = ctypes.c_void_p(0x10000)          # never dereferenced: validation fails first
    m = L.gs_map(fake, fake, fake, fake, 10)
    prm = _params()
    proj = L.gs_proj(10, *([fake] * (len(L.gs_proj._fields_) - 1)))
    P = ctypes.byref
    # null map / cameras / params
    assert lib.gs_project(None, fake, 1, P(prm), P(proj), fake, 1 << 20, None) == L.GS_ERR_NULL
    assert lib.gs_project(P(m), None, 1, P(prm), P(proj), fake, 1 << 20, None) == L.GS_ERR_NULL
    assert lib.gs_project(P(m), fake, 1, None, P(proj), fake, 1 << 20, None) == L.GS_ERR_NULL
    # bad counts
    assert lib.gs_project(P(m), fake, 0, P(prm), P(proj), fake, 1 << 20, None) == L.GS_ERR_ARG
    neg = L.gs_map(fake, fake, fake, fake, -1)
    assert lib.gs_project(P(neg), fake, 1, P(prm), P(proj), fake, 1 << 20, None) == L.GS_ERR_ARG
    # bad parameters
    for bad in (_params(tile_w=10), _params(tile_w=128, tile_h=2), _params(tile_w=16, tile_h=6), _params(tile_w=4, tile_h=16), _params(tile_w=16, tile_h=4), _params(near_plane=0.0), _params(alpha_max=0.0),
                _params(alpha_min=1.0), _params(eps2d=-1.0), _params(T_min=1.0), _params(guard=float("nan")),
                _params(ig_batch=3), _params(ig_batch=32), _params(fwd_batch=8), _params(fwd_batch=-1)):
        assert lib.gs_project(P(m), fake, 1, P(bad), P(proj), fake, 1 << 20, None) == L.GS_ERR_ARG
    # misaligned map pointer
    mis = L.gs_map(ctypes.c_void_p(0x10004), fake, fake, fake, 10)
    assert lib.gs_project(P(mis), fake, 1, P(prm), P(proj), fake, 1 << 20, None) == L.GS_ERR_ALIGN
    # workspace too small / misaligned
    assert lib.gs_project(P(m), fake, 1, P(prm), P(proj), fake, 8, None) == L.GS_ERR_WORKSPACE
    assert lib.gs_project(P(m), fake, 1, P(prm), P(proj), ctypes.c_void_p(0x10010), 1 << 20, None) == L.GS_ERR_ALIGN
    # bins capacity
    bins = L.gs_bins(0, 10, fake, fake, fake, fake)
    assert lib.gs_bin_sort(P(proj), fake, 1, P(prm), P(bins), fake, 1 << 30, None) == L.GS_ERR_ARG
    # the optional item order: aligned, with a capacity in [0, 2^32)
    bins = L.gs_bins(100, 10, fake, fake, fake, fake, ctypes.c_void_p(0x10002), 50)
    assert lib.gs_bin_sort(P(proj), fake, 1, P(prm), P(bins), fake, 1 << 30, None) == L.GS_ERR_ALIGN
    for cap in (-1, 1 << 32):
        bins = L.gs_bins(100, 10, fake, fake, fake, fake, fake, cap)
        assert lib.gs_bin_sort(P(proj), fake, 1, P(prm), P(bins), fake, 1 << 30, None) == L.GS_ERR_ARG
    # images: a misaligned output, saved image or image gradient is refused before any launch
    bins = L.gs_bins(100, 10, fake, fake, fake, fake)
    odd = ctypes.c_void_p(0x10002)
    img_bad = L.gs_image(fake, odd, None, fake, fake, None)
    assert lib.gs_render_fwd(P(m), P(proj), P(bins), fake, 1, P(prm), P(img_bad), None) == L.GS_ERR_ALIGN
    # the one-launch small render: size limits, a status word, aligned images
    img_ok = L.gs_image(fake, fake, None, fake, fake, None)
    big = L.gs_map(fake, fake, fake, fake, L.GS_SMALL_MAX_GAUSSIANS + 1)
    assert lib.gs_render_small(P(big), fake, 1, P(prm), P(img_ok), fake, None) == L.GS_ERR_ARG
    assert lib.gs_render_small(P(m), fake, L.GS_SMALL_MAX_VIEWS + 1, P(prm), P(img_ok), fake, None) == L.GS_ERR_ARG
    assert lib.gs_render_small(P(m), fake, 1, P(prm), P(img_ok), None, None) == L.GS_ERR_NULL
    assert lib.gs_render_small(P(m), fake, 1, P(prm), P(img_bad), fake, None) == L.GS_ERR_ALIGN
    assert lib.gs_render_small(P(m), fake, 1, P(_params(tile_w=12)), P(img_ok), fake, None) == L.GS_ERR_ARG
    img = L.gs_image(fake, fake, None, fake, fake, None)
    out = L.gs_map_grad(fake, fake, fake, fake)
    for fwd, grad in ((img_bad, L.gs_image_grad(fake, fake)), (img, L.gs_image_grad(odd, None)),
                      (img, L.gs_image_grad(None, odd))):
        assert lib.gs_render_bwd(P(m), P(proj), P(bins), P(fwd), P(grad), fake, 1, P(prm), P(out), fake, 1 << 30,
                                 None) == L.GS_ERR_ALIGN
    assert lib.gs_render_bwd_noalloc(P(m), P(proj), P(bins), P(img), P(L.gs_image_grad(odd, None)), fake, 1, P(prm),
                                     P(out), None) == L.GS_ERR_ALIGN
    # info gain: unknown mode, null output
    assert lib.gs_info_gain_batch(P(m), fake, 1, P(prm), 7, fake, fake, 0, 100, 10, fake, 1 << 30, None) == L.GS_ERR_ARG
    assert lib.gs_info_gain_batch(P(m), fake, 1, P(prm), 0, None, fake, 0, 100, 10, fake, 1 << 30, None) == L.GS_ERR_NULL
    assert lib.gs_info_gain_batch(P(m), fake, 1, P(prm), 0, fake, fake, -1, 100, 10, fake, 1 << 30, None) == L.GS_ERR_ARG
    # image loss: sizes, weights, depth pointers, workspace
    sz = (ctypes.c_int32 * 4)(64, 48, 37, 29)
    w = L.gs_loss_weights(1.0, 0.4, 0.1)
    nb = ctypes.c_size_t(0)
    assert lib.gs_image_loss_workspace_size(sz, 2, P(nb)) == L.GS_OK and nb.value % 256 == 0
    need = nb.value
    assert need >= 36 * (64 * 48 + 37 * 29)
    assert lib.gs_image_loss_workspace_size(sz, 1, P(nb)) == L.GS_OK and nb.value < need
    assert lib.gs_image_loss_workspace_size((ctypes.c_int32 * 2)(0, 5), 1, P(nb)) == L.GS_ERR_ARG
    assert lib.gs_image_loss_workspace_size(None, 1, P(nb)) == L.GS_ERR_NULL
    ok = (sz, 2, fake, fake, fake, fake, P(w), fake, fake, fake, fake, need, None)

    def call(**kw):
        a = list(ok)
        for i, v in kw.items():
            a[int(i[1:])] = v
        return lib.gs_image_loss(*a)
    assert call(a0=None) == L.GS_ERR_NULL and call(a2=None) == L.GS_ERR_NULL and call(a7=None) == L.GS_ERR_NULL
    assert call(a1=0) == L.GS_ERR_ARG
    assert call(a3=None, a5=None) == L.GS_ERR_NULL                   # w_depth != 0 needs depth
    assert call(a3=None) == L.GS_ERR_NULL                            # depth and depth_ref together
    for bad in ((-1.0, 0.4, 0.1), (1.0, float("nan"), 0.1), (1.0, 0.4, float("inf"))):
        assert call(a6=P(L.gs_loss_weights(*bad))) == L.GS_ERR_ARG
    assert call(a11=need - 256) == L.GS_ERR_WORKSPACE
    assert call(a8=ctypes.c_void_p(0x10002)) == L.GS_ERR_ALIGN
    # Adam step: tensor count, sizes, parameters, alignment
    ptrs = (ctypes.c_void_p * 2)(fake, fake)
    sizes = (ctypes.c_int64 * 2)(16, 8)
    ap = L.gs_adam_params(1e-3, 0.9, 0.999, 1e-8)
    assert lib.gs_adam_step(ptrs, ptrs, ptrs, ptrs, sizes, 0, P(ap), fake, None) == L.GS_ERR_ARG
    assert lib.gs_adam_step(ptrs, ptrs, ptrs, ptrs, sizes, 9, P(ap), fake, None) == L.GS_ERR_ARG
    assert lib.gs_adam_step(None, ptrs, ptrs, ptrs, sizes, 2, P(ap), fake, None) == L.GS_ERR_NULL
    assert lib.gs_adam_step(ptrs, ptrs, ptrs, ptrs, sizes, 2, P(ap), None, None) == L.GS_ERR_NULL
    assert lib.gs_adam_step(ptrs, ptrs, ptrs, ptrs, (ctypes.c_int64 * 2)(16, 6), 2, P(ap), fake, None) == L.GS_ERR_ARG
    for bad in ((-1.0, 0.9, 0.999, 1e-8), (1e-3, 1.0, 0.999, 1e-8), (1e-3, 0.9, 0.999, 0.0),
                (float("nan"), 0.9, 0.999, 1e-8)):
        assert lib.gs_adam_step(ptrs, ptrs, ptrs, ptrs, sizes, 2, P(L.gs_adam_params(*bad)), fake, None) == L.GS_ERR_ARG
    mis = (ctypes.c_void_p * 2)(fake, ctypes.c_void_p(0x10004))
    assert lib.gs_adam_step(mis, ptrs, ptrs, ptrs, sizes, 2, P(ap), fake, None) == L.GS_ERR_ALIGN
    # read_status: null
    f = ctypes.c_uint32(0)
    assert lib.gs_read_status(None, P(f)) == L.GS_ERR_NULL


def test_python_binding_raises_without_library(monkeypatch):
    monkeypatch.setattr(L, "LIB_PATH", "/nonexistent/libgs103.so")
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(L.GSError):
        L.lib()


def test_plain_c_program_builds_links_and_calls(lib, tmp_path):
    """The boundary is a C library: a C99 program (strict, warnings as errors) and the same
    source as C++11 compile against include/gs.h alone, and the C program links against
    libgs103.so and calls its host-side entry points without any Python or torch."""
    src = tmp_path / "use_gs.c"
    src.write_text("\n".join([
        "#include <stdio.h>",
        "#include \"gs.h\"",
        "int main(void) {",
        "  size_t b = 0;",
        "  gs_status s = gs_workspace_size(GS_OP_PROJECT, 1000, 4, 0, 0, 0, &b);",
        "  gs_status bad = gs_workspace_size(GS_OP_PROJECT, -1, 4, 0, 0, 0, &b);",
        "  printf(\"%d %d %zu|%s|%s\\n\", (int)s, (int)bad, b, gs_status_str(bad), gs_version());",
        "  return s == GS_OK && bad == GS_ERR_ARG && b > 0 ? 0 : 1;",
        "}"]) + "\n")
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(L.LIB_PATH)
    subprocess.check_call(["g++", "-std=c++11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, "-x", "c++",
                           str(src), "-c", "-o", str(tmp_path / "use_gs_cxx.o")])
    exe = tmp_path / "use_gs"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(src),
                           "-L", libdir, "-lgs103", "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    codes, status, version = out.stdout.strip().split("|")
    assert codes.split()[:2] == [str(L.GS_OK), str(L.GS_ERR_ARG)]
    assert status.startswith("GS_ERR_ARG") and version
