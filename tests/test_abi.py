"""The C-ABI library builds, loads without a GPU and exports every entry
point the header declares; host-side marshalling checks."""
import ctypes as C
import os
import re

import pytest

import paper_2608_03695_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mslice_[a-z_]+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return C.CDLL(pkg.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(pkg.EXPORTS) == names


def test_default_opts_and_error_string(lib):
    o = pkg.default_opts()
    assert (o.n_iterations, o.K, o.max_rounds, o.max_levels, o.stop_level) == (2, 4, 100, 32, -1)
    assert (o.gamma_num, o.gamma_den, o.omega_num, o.omega_den) == (1, 1, 1, 1)
    L = pkg.lib()
    assert L.mslice_last_error() == b""


def test_host_side_rejections_need_no_gpu():
    L = pkg.lib()
    h = C.c_void_p()
    # T < 1 and a null handle are rejected before any CUDA call
    assert L.mslice_build(None, 0, 0, 1, 1, C.byref(h)) == pkg.MSLICE_EINVAL
    assert L.mslice_info(None, None, None, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_leiden_ex(None, None, None, None, None, None) == pkg.MSLICE_EINVAL
    assert b"handle" in L.mslice_last_error()
    L.mslice_free(None)
    # batch entry points: null batches are rejected before any CUDA call
    assert L.mslice_batch_add(None, None, 1, 1, 1, 1, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_batch_run(None, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_batch_results(None, 0, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_batch_info(None, None, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_batch_clear(None) == pkg.MSLICE_EINVAL
    assert L.mslice_batch_kernel_launches(None) == -1
    assert L.mslice_batch_create(0, None, None) == pkg.MSLICE_EINVAL
    L.mslice_batch_free(None)
    # server entry points
    assert L.mslice_server_create(None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_server_add_graph(None, 10, None) == pkg.MSLICE_EINVAL
    assert L.mslice_server_submit(None, 0, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_server_wait(None, 1, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_server_window_info(None, 0, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_server_window_read(None, 0, 0, None, None, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_server_window_restore(None, 0, None, 0, None) == pkg.MSLICE_EINVAL
    L.mslice_server_free(None)
    # general forms and windowed optimisation: null handles, bad windows
    assert L.mslice_leiden_general(None, None, None, None, None, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_modularity_general(None, None, None, None, None) == pkg.MSLICE_EINVAL
    assert L.mslice_batch_add_general(None, None, 1, 1, 1, 1, None, None, None) == pkg.MSLICE_EINVAL
    from paper_2608_03695_gb300 import synth
    snaps = synth.random_temporal(5, 6, p=0.4, seed=1)
    for W, S in [(0, 1), (3, 0), (3, 3)]:
        with pytest.raises(pkg.MsliceError) as e:
            pkg.leiden_windowed(snaps, W, S)
        assert e.value.code == pkg.MSLICE_EINVAL
    o = pkg.ServerOpts()
    L.mslice_server_default_opts(C.byref(o))
    assert (o.window, o.n_slots, o.max_batch, o.hbm_budget, o.max_batch_nodes) == (8, 2, 64, 0, 1 << 21)
    assert (o.solve.n_iterations, o.solve.K, o.solve.stop_level) == (2, 4, -1)


def test_struct_layouts_match_header():
    # field order and sizes of the ctypes mirrors follow include/mslice.h
    assert C.sizeof(pkg.Csr) == 32
    assert C.sizeof(pkg.ServerOpts) == 16 + 8 + 8 + 32 + C.sizeof(pkg.Opts)
    assert C.sizeof(pkg.RequestInfo) == 8 + 8 + 8 + 24 + 8 + 8 + 16
    assert C.sizeof(pkg.Opts) == 4 * 4 + 8 + 4 * 8 + 4 * 4 + 4 * 4 + 2 * 8
    assert C.sizeof(pkg.Stats) == 4 + 4 + 8 * 7 + 8 + 4 + 4 + 8 + 8 * 5 + 8 * 3 + 4 * 4 + 8 * 4


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Sizes and field offsets of every ABI struct, as gcc lays them out from
    include/mslice.h, equal the ctypes mirrors of the binding."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    mirrors = {"mslice_csr": pkg.Csr, "mslice_opts": pkg.Opts, "mslice_stats": pkg.Stats,
               "mslice_server_opts": pkg.ServerOpts, "mslice_request_info": pkg.RequestInfo,
               "mslice_general": pkg.General}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mslice.h"', 'int main(void) {']
    for cname, cls in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, cls in mirrors.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_header_constants_match_the_binding():
    """Every MSLICE_* status code and flag the header defines has the same
    value in the Python binding."""
    text = open(os.path.join(ROOT, "include", "mslice.h")).read()
    defs = dict(re.findall(r"#define\s+(MSLICE_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text))
    defs.update(re.findall(r"(MSLICE_[A-Z]+)\s*=\s*(\d+)", text))  # enum members
    assert {"MSLICE_DEVICE_PTRS", "MSLICE_PROFILE", "MSLICE_AUTOTUNE", "MSLICE_NULL_GLOBAL"} <= set(defs)
    for name, value in defs.items():
        assert getattr(pkg, name) == int(value), name
    flags = [int(defs[k]) for k in ("MSLICE_DEVICE_PTRS", "MSLICE_PROFILE", "MSLICE_AUTOTUNE", "MSLICE_NULL_GLOBAL")]
    assert all(f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)  # distinct single bits
