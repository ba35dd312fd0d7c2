"""The C ABI library loads and exports every function include/tsgne.h declares
(no GPU needed: nothing here launches a kernel)."""

import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import paper_2310_11186_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsgne.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tsgne_[a-zA-Z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_2310_11186_gb300 import build

    build.build()
    return pkg.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("tsgne_build_P", "tsgne_step", "tsgne_run", "tsgne_kl"):
        assert must in names


def test_library_exports_every_declared_symbol(built):
    raw = ctypes.CDLL(pkg.library_path)
    for name in _declared():
        assert hasattr(raw, name), name
    # the binding declares exactly the same set
    assert sorted(pkg.EXPORTS) == _declared()


def test_host_only_calls(built):
    c = pkg.tsgne_config_default()
    assert c.perplexity == 30.0 and c.ee_iters == 250 and c.early_exag == 12.0
    assert abs(c.momentum0 - 0.5) < 1e-7 and abs(c.momentum1 - 0.8) < 1e-7
    assert pkg.tsgne_status_string(2) == "TSGNE_ERR_BAD_CSR"
    assert isinstance(pkg.tsgne_last_error(None), str)
    with pytest.raises(pkg.TsgneError) as ei:
        pkg.tsgne_create(pkg.tsgne_config_default(perplexity=1.0))
    assert ei.value.status == 1


@pytest.mark.parametrize("bad", [
    dict(spin_budget_cycles=0), dict(spin_budget_cycles=-5), dict(repulsion=2), dict(theta=-0.1),
    dict(theta=1.5), dict(precision=2), dict(p_walks=513), dict(p_walks=-1), dict(p_walk_length=0),
    dict(p_walk_length=65), dict(k_nn=257), dict(min_gain=-1.0),
])
def test_invalid_configurations_are_rejected_before_device_work(built, bad):
    with pytest.raises(pkg.TsgneError) as ei:
        pkg.tsgne_create(pkg.tsgne_config_default(**bad))
    assert ei.value.status == 1  # INVALID_ARG, no CUDA call needed to decide it


def test_noalloc_rejects_bad_arguments_before_device_work(built):
    """tsgne_repulsion_noalloc checks sizes and pointer alignment before it
    touches the GPU (these pointers are never dereferenced), and says why
    through tsgne_last_error(NULL)."""
    lib = pkg.lib()
    f = lib.tsgne_repulsion_noalloc
    vp = ctypes.c_void_p
    # Y misaligned by 4 bytes (a float pair at an odd float offset)
    assert f(100, vp(0x100004), vp(0x200000), vp(0x300000), None) == 1
    assert "aligned" in lib.tsgne_last_error(None).decode()
    assert f(100, vp(0x100000), vp(0x200002), vp(0x300000), None) == 1
    assert f(100, vp(0x100000), vp(0x200000), vp(0x300004), None) == 1
    # too many points, then too few
    assert f(pkg.NOALLOC_MAX_N + 1, vp(0x100000), vp(0x200000), vp(0x300000), None) == 1
    assert "maximum" in lib.tsgne_last_error(None).decode()
    assert f(1, vp(0x100000), vp(0x200000), vp(0x300000), None) == 1
    assert f(100, None, vp(0x200000), vp(0x300000), None) == 1


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "library_path", "/nonexistent/libtsgne.so")
    with pytest.raises(RuntimeError):
        pkg.lib()


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c++", "c++11")])
def test_header_is_valid_plain_c_and_cpp(tmp_path, lang, std):
    """The boundary is a C ABI: the header compiles as strict C99 (and as
    C++11) with every warning an error, and its entry points can be called."""
    cc = shutil.which("gcc") if lang == "c" else shutil.which("g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / "use.c"
    src.write_text(
        '#include "tsgne.h"\n'
        "int main(void) {\n"
        "  tsgne_config c;\n"
        "  tsgne_config_default(&c);\n"
        "  tsgne_ctx* ctx = 0;\n"
        "  tsgne_status s = tsgne_create(&ctx, &c, 0);\n"
        "  if (s == TSGNE_OK) tsgne_destroy(ctx);\n"
        "  return tsgne_server_estimate_bytes(1000, 6000, 2) > 0 ? 0 : 1;\n"
        "}\n")
    r = subprocess.run([cc, "-x", lang, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.dirname(HEADER), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_a_c_program_links_and_calls_the_library(built, tmp_path):
    """A plain C program links against libtsgne.so and calls the host-only
    entry points (no GPU needed for these)."""
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / "main.c"
    src.write_text(
        '#include <string.h>\n#include "tsgne.h"\n'
        "int main(void) {\n"
        "  tsgne_config c;\n"
        "  tsgne_config_default(&c);\n"
        "  if (c.perplexity != 30.0f || c.repulsion != 0 || c.spin_budget_cycles <= 0) return 1;\n"
        "  if (strcmp(tsgne_status_string(TSGNE_ERR_TIMEOUT), \"TSGNE_ERR_TIMEOUT\") != 0) return 2;\n"
        "  c.perplexity = 1.0f;\n"
        "  tsgne_ctx* ctx = 0;\n"
        "  if (tsgne_create(&ctx, &c, 0) != TSGNE_ERR_INVALID_ARG || ctx != 0) return 3;\n"
        "  return tsgne_server_estimate_bytes(1000, 6000, 2) > 0 ? 0 : 4;\n"
        "}\n")
    libdir = os.path.dirname(pkg.library_path)
    exe = tmp_path / "main"
    r = subprocess.run([cc, "-std=c99", str(src), "-I", os.path.dirname(HEADER), "-L", libdir, "-ltsgne",
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)


def test_outputs_of_the_wrong_size_are_refused_before_the_library_writes(built):
    # _out runs before any call into the library: a short or long buffer never
    # reaches it
    with pytest.raises(ValueError):
        pkg._out(10, np.zeros((9, 2), np.float32))
    with pytest.raises(ValueError):
        pkg._out(10, np.zeros(21, np.float32))
    with pytest.raises(ValueError):  # a dtype that would need a copy
        pkg._out(10, np.zeros((10, 2), np.float64))
    out, buf = pkg._out(10, np.zeros((10, 2), np.float32))
    assert out.shape == (10, 2) and buf[2] is out
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    with pytest.raises(ValueError):
        pkg.tsgne_shortest_path_embedding(rp, col, np.array([0], np.int32), out=np.zeros((2, 2), np.float32))


def test_inputs_of_the_wrong_size_are_refused_before_the_library_reads(built):
    rp = np.array([0, 2, 3, 4], np.int64)
    pkg._graph(3, rp, np.array([1, 2, 0, 0], np.int32))
    with pytest.raises(ValueError):  # col shorter than row_ptr[n]
        pkg._graph(3, rp, np.array([1, 2, 0], np.int32))
    with pytest.raises(ValueError):  # row_ptr of the wrong length
        pkg._graph(4, rp, np.array([1, 2, 0, 0], np.int32))
    pkg._rows(np.zeros((3, 2), np.float32), 3, 2, "Y0")
    with pytest.raises(ValueError):
        pkg._rows(np.zeros((2, 2), np.float32), 3, 2, "Y0")
    with pytest.raises(ValueError):  # X with the wrong row count, before any call into the library
        pkg.tsgne_build_P(None, 3, rp, np.array([1, 2, 0, 0], np.int32), np.zeros((2, 4), np.float32))
    with pytest.raises(ValueError):  # P with the wrong length
        pkg.tsgne_set_P(None, 3, rp, np.array([1, 2, 0, 0], np.int32), np.zeros(3, np.float32))
