"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gsplat103.h declares; host-only entry points behave as documented.
No kernel is launched here (these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2312_02121_gb300 import build as gsbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gsplat103.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(gs_[a-z0-9_]+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_02121_gb300 import binding
    gsbuild.build()
    return binding.load()


def test_header_declares_the_five_stages():
    fns = declared_functions()
    for name in ("gs_project", "gs_bin_and_sort", "gs_rasterize_fwd", "gs_rasterize_bwd", "gs_project_bwd"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2312_02121_gb300 import binding
    assert sorted(binding.SIGNATURES) == declared_functions()


def test_version_and_struct_sizes(lib):
    from paper_2312_02121_gb300 import binding
    assert binding.gs_version() == 200
    assert ctypes.sizeof(binding.GsView) == 120


def test_views_layout(lib):
    from paper_2312_02121_gb300 import binding
    from paper_2312_02121_gb300 import workloads as wl
    cams = [wl.camera_at_distance(3.0, 40, 20, 50.0), wl.camera_at_distance(3.0, 16, 16, 50.0),
            wl.camera_at_distance(3.0, 33, 17, 50.0)]
    v = binding.Views(cams, [(0, 10), (10, 0), (10, 5)], device="cpu")
    assert (v.V, v.P, v.T, v.pixels) == (3, 15, 3 * 2 + 1 + 3 * 2, 800 + 256 + 561)
    assert [v.host[i].proj_offset for i in range(3)] == [0, 10, 10]
    assert [v.host[i].tile_offset for i in range(3)] == [0, 6, 7]
    assert [v.host[i].pixel_offset for i in range(3)] == [0, 800, 1056]
    assert [(v.host[i].tiles_x, v.host[i].tiles_y) for i in range(3)] == [(3, 2), (1, 1), (3, 2)]


def test_views_layout_rejects_bad_sizes(lib):
    from paper_2312_02121_gb300 import binding
    from paper_2312_02121_gb300 import workloads as wl
    cam = wl.camera_at_distance(3.0, 0, 20, 50.0)
    with pytest.raises(binding.GsError) as e:
        binding.Views([cam], [(0, 1)], device="cpu")
    assert e.value.code == binding.GS_ERR_INVALID_ARG


def test_workspace_sizes_grow_with_capacity(lib):
    from paper_2312_02121_gb300 import binding
    a = binding.gs_bin_and_sort_workspace_size(1000, 10_000, 64)
    b = binding.gs_bin_and_sort_workspace_size(1000, 20_000, 64)
    assert 0 < a < b and a % 256 == 0
    assert binding.gs_rasterize_bwd_workspace_size(1000, True) >= 1000 * 9 * 4
    assert binding.gs_rasterize_bwd_workspace_size(1000, False) == 0


def test_invalid_arguments_are_rejected_on_the_host(lib):
    # null pointers / negative sizes return GS_ERR_INVALID_ARG before any CUDA call
    assert lib.gs_project(None, 1, 10, None, None, None, 0.3, None, None, None, None, None, None, None) == 1
    assert b"null pointer" in lib.gs_last_error()
    assert lib.gs_project(None, -1, 10, None, None, None, 0.3, None, None, None, None, None, None, None) == 1
    assert lib.gs_rasterize_fwd(None, 0, 4, None, None, None, None, None, None, None, None, None, None, None,
                                None, None) == 1
    assert lib.gs_tile_order(None, 5, None, 0, None, None) == 1
    assert lib.gs_bin_and_sort(None, 1, 10, 4, None, None, None, 100, None, 0, None, None, None, None, None, None,
                               None) == 1
    assert lib.gs_project_bwd(None, 1, -5, None, None, None, 0.3, None, None, None, None, None, None, None,
                              None) == 1


def test_bin_and_sort_rejects_a_misaligned_workspace(lib):
    # fake (never dereferenced) addresses: every check before the first CUDA call passes except the
    # workspace alignment
    from paper_2312_02121_gb300 import binding
    P, cap, T = 10, 100, 4
    need = binding.gs_bin_and_sort_workspace_size(P, cap, T)
    fake = 1 << 20
    args = (fake, 1, P, T, fake, fake, fake, cap)
    outs = (fake, None, None, fake, fake, fake, None)
    assert lib.gs_bin_and_sort(*args, fake + 8, need, *outs) == binding.GS_ERR_INVALID_ARG
    assert b"16-byte alignment" in lib.gs_last_error()
    assert lib.gs_bin_and_sort(*args, fake, need - 1, *outs) == binding.GS_ERR_INVALID_ARG
    assert b"workspace of" in lib.gs_last_error()


def test_static_scratch_covers_the_static_limits(lib):
    # at the documented limits the workspace check passes; the call then fails only at its first CUDA
    # call (there is no GPU here), not with "needs ... bytes of scratch"
    import re
    hdr = open(HEADER).read()
    P = int(re.search(r"#define GS_STATIC_MAX_PROJECTIONS (\d+)", hdr).group(1))
    K = int(re.search(r"#define GS_STATIC_MAX_INTERSECTIONS (\d+)", hdr).group(1))
    fake = 1 << 20
    rc = lib.gs_bin_and_sort_static(fake, 1, P, 65536, fake, fake, fake, K, fake, None, None, fake, fake, fake, None)
    assert b"bytes of scratch" not in lib.gs_last_error(), lib.gs_last_error()
    assert rc != 0  # no device in this container


def test_raster_config_rejects_a_wrong_warp_hits_buffer(lib):
    # the forward-to-backward hand-off takes device int32 words; anything else is refused on the host
    import torch
    from paper_2312_02121_gb300 import binding
    with pytest.raises(TypeError):
        binding.RasterConfig(device="cpu", warp_hits=torch.zeros(8, dtype=torch.uint8))
    with pytest.raises(TypeError):
        binding.RasterConfig(device="cpu", warp_hits=torch.zeros(8, dtype=torch.int32))  # host memory
    cfg = binding.RasterConfig(device="cpu")
    assert cfg.describe()["warp_hits"] is False and cfg.c.warp_hits is None



def _kind_of_c(t: str):
    """'ptr', 'char*', or (int|float, bytes) of a C type written in the header."""
    t = " ".join(t.replace("const", " ").split())
    if "*" in t:
        return "char*" if t.replace(" ", "") == "char*" else "ptr"
    sizes = {"int": 4, "int32_t": 4, "int64_t": 8, "size_t": 8, "float": 4, "double": 8}
    return ("float" if t in ("float", "double") else "int", sizes[t])


def _kind_of_ctypes(c):
    if c is ctypes.c_char_p:
        return "char*"
    if c is ctypes.c_void_p:
        return "ptr"
    return ("float" if c in (ctypes.c_float, ctypes.c_double) else "int", ctypes.sizeof(c))


def _param_type(param: str) -> str:
    """The type of one 'type name' parameter (the name dropped, any stars kept)."""
    return re.sub(r"\b[A-Za-z_]\w*\s*$", "", param.strip()).strip()


def test_binding_signatures_match_the_header_prototypes():
    # every argument's kind (pointer, or integer / floating point of its width) and every return
    # type, read from the prototypes, against the ctypes declarations the binding installs
    from paper_2312_02121_gb300 import binding
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = re.findall(r"^\s*((?:const\s+)?[A-Za-z_]\w*\s*\**)\s*(gs_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text, re.M)
    assert sorted(name for _, name, _ in protos) == declared_functions()
    for ret, name, params in protos:
        params = " ".join(params.split())
        want = [] if params in ("", "void") else [_kind_of_c(_param_type(q)) for q in params.split(",")]
        res, argtypes = binding.SIGNATURES[name]
        assert [_kind_of_ctypes(a) for a in argtypes] == want, name
        assert _kind_of_ctypes(res) == _kind_of_c(ret), name


def test_binding_structs_match_the_header_layout(tmp_path):
    # the C compiler's offsetof / sizeof of every field of every struct the header declares,
    # against the ctypes structures the binding passes (host gcc: the layout is the platform's C ABI)
    import shutil
    import subprocess
    from paper_2312_02121_gb300 import binding
    cc = shutil.which(os.environ.get("CC", "gcc"))
    if cc is None:
        pytest.skip("no C compiler")
    structs = [binding.GsCamera, binding.GsView, binding.GsRasterConfig, binding.GsAdamConfig, binding.GsTuning]
    lines = ["#include <stdio.h>", '#include "gsplat103.h"', "int main(void) {"]
    for S in structs:
        n = S.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in S._fields_:
            lines.append(f'printf("{n} {f} %zu %zu\\n", offsetof({n}, {f}), sizeof((({n}*)0)->{f}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        f = ln.split()
        got[(f[0], f[1])] = tuple(int(x) for x in f[2:])
    for S in structs:
        n = S.__name__
        assert got[(n, "size")] == (ctypes.sizeof(S),), n
        for f, _ in S._fields_:
            d = getattr(S, f)
            assert got[(n, f)] == (d.offset, d.size), f"{n}.{f}"


def test_binding_constants_match_the_header_defines():
    from paper_2312_02121_gb300 import binding
    text = open(HEADER).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (GS_\w+) (\d+)u?\b", text, re.M)}
    assert {"GS_OK", "GS_ERR_INVALID_ARG", "GS_ERR_CAPACITY", "GS_FLAG_CAPACITY", "GS_TILE"} <= set(defines)
    for name, value in defines.items():
        if hasattr(binding, name):
            assert getattr(binding, name) == value, name


def test_every_entry_point_rejects_null_arguments_before_any_cuda_call(lib):
    # All pointers NULL, sizes small and positive: each compute entry point answers
    # GS_ERR_INVALID_ARG with a message naming itself, from its host checks (no GPU here, so a
    # call that reached CUDA first would answer GS_ERR_CUDA instead).
    from paper_2312_02121_gb300 import binding
    checked = 0
    for name, (res, argtypes) in binding.SIGNATURES.items():
        if res is not ctypes.c_int or not argtypes:
            continue
        args = [None if a is ctypes.c_void_p else 0.3 if a in (ctypes.c_float, ctypes.c_double)
                else (1 << 20) if a is ctypes.c_size_t else 16 for a in argtypes]
        rc = getattr(lib, name)(*args)
        msg = lib.gs_last_error().decode()
        assert rc == binding.GS_ERR_INVALID_ARG, (name, rc, msg)
        assert msg.startswith(name + ":"), (name, msg)
        checked += 1
    assert checked >= 18


def test_every_entry_point_rejects_a_negative_size_on_the_host(lib):
    # Each integer argument set to -1 in turn (boolean flags aside), every pointer aimed at a zeroed
    # host buffer: each compute entry point answers GS_ERR_INVALID_ARG from its host checks.
    from paper_2312_02121_gb300 import binding
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = {name: params for _, name, params in re.findall(
        r"^\s*((?:const\s+)?[A-Za-z_]\w*\s*\**)\s*(gs_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text, re.M)}
    buf = (ctypes.c_char * (1 << 20))()
    base = (ctypes.addressof(buf) + 255) & ~255
    checked = 0
    for name, (res, argtypes) in binding.SIGNATURES.items():
        if res is not ctypes.c_int or not argtypes:
            continue
        pnames = [re.findall(r"\w+", p)[-1] for p in protos[name].split(",")]
        for k, a in enumerate(argtypes):
            if a not in (ctypes.c_int32, ctypes.c_int64) or pnames[k] == "deterministic":
                continue
            args = [base if t is ctypes.c_void_p else 0.3 if t in (ctypes.c_float, ctypes.c_double)
                    else (1 << 19) if t is ctypes.c_size_t else (-1 if i == k else 1) for i, t in enumerate(argtypes)]
            rc = getattr(lib, name)(*args)
            assert rc == binding.GS_ERR_INVALID_ARG, (name, pnames[k], rc, lib.gs_last_error())
            checked += 1
    assert checked >= 40


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c++", "c++11")])
def test_header_is_clean_c99_and_cxx11(tmp_path, lang, std):
    # the boundary is consumable from plain C and from C++, without warnings under -pedantic
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("probe.c" if lang == "c" else "probe.cpp")
    src.write_text('#include "gsplat103.h"\nint main(void) { GsView v; v.g_count = GS_TILE; return v.g_count == 0; }\n')
    subprocess.run([cc, f"-std={std}", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.dirname(HEADER),
                    "-c", str(src), "-o", str(tmp_path / "probe.o")], check=True)


def test_views_exclusive_only_when_no_gaussian_is_shared():
    # gs_project_bwd_exclusive applies when the views' Gaussian ranges do not overlap (empty views
    # aside); the binding decides this on the host copy of the view table
    from paper_2312_02121_gb300 import binding
    from paper_2312_02121_gb300 import workloads as wl
    cam = wl.camera_at_distance(3.0, 40, 20, 50.0)
    mk = lambda ranges: binding.Views([cam] * len(ranges), ranges, device="cpu")
    assert binding.views_exclusive(mk([(0, 10)]))
    assert binding.views_exclusive(mk([(10, 5), (0, 10), (15, 0)]))
    assert binding.views_exclusive(mk([(0, 10), (10, 0), (20, 3)]))
    assert not binding.views_exclusive(mk([(0, 10), (9, 3)]))
    assert not binding.views_exclusive(mk([(0, 10), (0, 10)]))
