"""CPU checks of the C interface: the library loads, exports every function
that the headers under include/ declare, and the binding's struct layouts
match the C compiler's.  No compute call is made (there may be no GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))


def _declared():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:lbm_status|const char \*)\s*(lbm_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1503_06869_gb300 import _build, lbm
    _build.build()
    return lbm.load()


def test_header_declares_the_interface():
    names = _declared()
    for n in ("lbm_create", "lbm_create_batch", "lbm_set_particles", "lbm_step", "lbm_get_forces",
              "lbm_get_fields", "lbm_get_links", "lbm_destroy", "lbm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1503_06869_gb300 import lbm
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_\w+)", out))
    for n in _declared():
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(_declared()) <= set(lbm.SIGNATURES)


def test_struct_layouts_match_c(tmp_path):
    from paper_1503_06869_gb300 import lbm
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_grid_desc),'
                    ' sizeof(lbm_particle), sizeof(lbm_info), offsetof(lbm_grid_desc, prec),'
                    ' offsetof(lbm_particle, cell), offsetof(lbm_info, device_bytes));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    assert got == [C.sizeof(lbm.lbm_grid_desc), C.sizeof(lbm.lbm_particle), C.sizeof(lbm.lbm_info),
                   lbm.lbm_grid_desc.prec.offset, lbm.lbm_particle.cell.offset,
                   lbm.lbm_info.device_bytes.offset]


def test_status_strings_without_gpu(lib):
    assert lib.lbm_status_string(0) == b"ok"
    assert lib.lbm_status_string(1) == b"invalid argument"


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    """Descriptor validation happens on the host, before any CUDA call."""
    from paper_1503_06869_gb300 import lbm
    from lbm_inputs import shear_lattice
    h = C.c_void_p()
    assert lib.lbm_create(None, C.byref(h)) == lbm.LBM_ERR_ARG
    for mutate in (lambda d: setattr(d, "nx", 2), lambda d: setattr(d, "tau", 0.5),
                   lambda d: setattr(d, "magic", 0.0), lambda d: setattr(d, "rho0", -1.0),
                   lambda d: d.wall_u_hi.__setitem__(0, 0.2), lambda d: setattr(d, "prec", 9)):
        d = lbm.grid_desc(shear_lattice(8, 8, 8, 0.8, 0.01))
        mutate(d)
        assert lib.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_ERR_ARG
        assert not h.value
    assert lib.lbm_create_batch(None, 0, C.byref(h)) == lbm.LBM_ERR_ARG


def test_null_context_is_rejected(lib):
    from paper_1503_06869_gb300 import lbm
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_destroy(None) == lbm.LBM_ERR_ARG
    assert lib.lbm_last_error(None) == b"null context"


def test_free_slip_descriptor_rules_without_gpu(lib):
    """A free-slip axis cannot be periodic, and free-slip y walls cannot move
    (the moving walls of Sec. 4 are no-slip); both are refused on the host."""
    from paper_1503_06869_gb300 import lbm
    from lbm_inputs import shear_lattice
    h = C.c_void_p()
    d = lbm.grid_desc(shear_lattice(8, 8, 8, 0.8, 0.01))
    d.free_slip[0] = 1                      # x is periodic in the shear lattice
    assert lib.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_ERR_ARG and not h.value
    d = lbm.grid_desc(shear_lattice(8, 8, 8, 0.8, 0.01))
    d.free_slip[1] = 1                      # y walls move at -/+ uw
    assert lib.lbm_create(C.byref(d), C.byref(h)) == lbm.LBM_ERR_ARG and not h.value


@pytest.mark.parametrize("M,N,nq,mu", [(0, 5, 24, 1.0), (65, 5, 24, 1.0), (2, 1, 24, 1.0), (2, 11, 24, 1.0),
                                       (2, 5, 1, 1.0), (2, 5, 65, 1.0), (2, 5, 24, 0.0), (2, 5, 24, float("nan"))])
def test_slender_body_sizes_are_checked_before_touching_the_gpu(lib, M, N, nq, mu):
    from paper_1503_06869_gb300 import lbm
    h = C.c_void_p()
    assert lib.lbm_sbf_create(M, N, nq, mu, None, C.byref(h)) == lbm.LBM_ERR_ARG
    assert not h.value
    assert lib.lbm_sbf_create(2, 5, 24, 1.0, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_sbf_destroy(None) == lbm.LBM_ERR_ARG


def test_a_c_program_links_and_calls_the_library(lib, tmp_path):
    """The headers compile as C99 with warnings as errors and a C program
    links against the shared library and gets its host-side answers (no
    call that needs a device)."""
    from paper_1503_06869_gb300 import lbm
    prog = tmp_path / "use.c"
    prog.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "lbm.h"
#include "lbm_sbf.h"
int main(void) {
    lbm_ctx *c = NULL;
    lbm_sbf *s = NULL;
    lbm_grid_desc d;
    memset(&d, 0, sizeof d);
    d.nx = 2; d.ny = 8; d.nz = 8; d.tau = 0.8; d.magic = 3.0 / 16.0; d.rho0 = 1.0;
    if (lbm_create(&d, &c) != LBM_ERR_ARG || c) return 1;
    if (lbm_create(NULL, &c) != LBM_ERR_ARG) return 2;
    if (lbm_sbf_create(0, 5, 24, 1.0, NULL, &s) != LBM_ERR_ARG || s) return 3;
    if (lbm_destroy(NULL) != LBM_ERR_ARG || lbm_sbf_destroy(NULL) != LBM_ERR_ARG) return 4;
    if (strcmp(lbm_status_string(LBM_ERR_ARG), "invalid argument") != 0) return 5;
    if (strcmp(lbm_last_error(NULL), "null context") != 0) return 6;
    puts("ok");
    return 0;
}
''')
    exe = tmp_path / "use"
    libdir = os.path.dirname(lbm.LIB_PATH)
    name = os.path.basename(lbm.LIB_PATH)[3:-3]
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(prog), "-o", str(exe), "-L", libdir, f"-l{name}", f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


def test_the_c_usage_example_compiles_and_links(lib, tmp_path):
    """The C usage example (tests/c_usage_example.c, also shown in the
    project's readme) builds against the headers and the library (it is not
    run: it needs a GPU)."""
    from paper_1503_06869_gb300 import lbm
    prog = os.path.join(ROOT, "tests", "c_usage_example.c")
    libdir = os.path.dirname(lbm.LIB_PATH)
    name = os.path.basename(lbm.LIB_PATH)[3:-3]
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    prog, "-o", str(tmp_path / "example"), "-L", libdir, f"-l{name}",
                    f"-Wl,-rpath,{libdir}"], check=True)


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the built library the binding raises."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1503_06869_gb300 import lbm\n"
            "try:\n    lbm.load(%r)\nexcept ImportError as e:\n    print('raised', e)\n") % (
        ROOT, str(tmp_path / "liblbm_missing.so"))
    r = subprocess.run([os.sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("raised CUDA library not built"), (r.stdout, r.stderr)


def test_the_package_never_reaches_the_oracle():
    """The product package imports nothing from oracle/ (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1503_06869_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M), f
                assert "lbm_oracle" not in src, f


def test_the_oracle_never_reaches_the_package():
    """The oracle shares no code with the CUDA library: it neither imports the
    package nor includes its headers or sources."""
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(odir, f)).read()
            assert not re.search(r"^\s*(from|import)\s+paper_1503_06869_gb300\b", src, flags=re.M), f
            assert not re.search(r'#include\s+"(lbm\.h|lbm_sbf\.h|lbm_internal\.cuh)"', src), f
            assert "csrc" not in src, f
