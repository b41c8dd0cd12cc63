"""The C-ABI library builds, loads without a GPU and exports every symbol
declared in include/hf.h; the binding's declarations match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hf_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1303_4916_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ["hf_basis_create", "hf_schwarz", "hf_fock_jk", "hf_scf_solve", "hf_serve_submit",
                     "hf_serve_poll", "hf_strerror", "hf_ctx_create"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1303_4916_gb300 import _abi
    assert set(_abi.SIGNATURES) == set(declared_functions())


def test_strerror_and_defaults_without_gpu(lib):
    from paper_1303_4916_gb300 import _abi
    L = _abi.load()
    assert L.hf_strerror(_abi.HF_ERR_ODD_ELECTRONS) == b"odd electron count"
    o = _abi.hf_scf_opts()
    L.hf_scf_opts_default(ctypes.byref(o))
    assert o.max_iter == 128 and o.e_tol == 1e-8 and o.diis_size == 8
    assert o.jk.schwarz_tau == 1e-12 and o.jk.fp32_bound == 0.0


def test_ctx_create_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1303_4916_gb300 import _abi
    L = _abi.load()
    h = ctypes.c_void_p()
    rc = L.hf_ctx_create(ctypes.byref(h), 0, 0, None)
    assert rc == _abi.HF_ERR_CUDA
    assert not h.value


def test_generated_header_is_current():
    import subprocess
    import sys
    import tempfile
    gen = os.path.join(ROOT, "paper_1303_4916_gb300", "csrc", "gen_eri.py")
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "x.cuh")
        subprocess.run([sys.executable, gen, out, "2"], check=True)
        assert open(out).read() == open(os.path.join(ROOT, "paper_1303_4916_gb300", "csrc",
                                                      "eri_classes.cuh")).read()


def test_binding_constants_match_header():
    """Every integer #define of the header (status codes, flags, sizes) has
    the same value in the binding."""
    from paper_1303_4916_gb300 import _abi
    defs = {}
    for h in HEADERS:
        for m in re.finditer(r"^#define\s+(HF_\w+)\s+\(?(-?\d+)u?\)?", open(h).read(), flags=re.M):
            defs[m.group(1)] = int(m.group(2))
    assert len(defs) > 15
    for name, v in defs.items():
        if hasattr(_abi, name):
            assert getattr(_abi, name) == v, name
    for name in ("HF_OK", "HF_PENDING", "HF_ERR_INVALID", "HF_ERR_TOO_LARGE", "HF_JK_DF64", "HF_JK_HOST",
                 "HF_JK_FP32_BOYS", "HF_NCLASS"):
        assert hasattr(_abi, name) and name in defs, name


def test_jk_opts_sets_the_header_flags(lib):
    import paper_1303_4916_gb300 as hf
    from paper_1303_4916_gb300 import _abi
    d = hf.jk_opts()
    assert d.schwarz_tau == 1e-12 and d.fp32_bound == 0.0 and d.flags == 0
    o = hf.jk_opts(schwarz_tau=0.0, fp32_bound=1e-5, host=True, fp32_boys=True, df64=True)
    assert o.schwarz_tau == 0.0 and o.fp32_bound == 1e-5
    assert o.flags == _abi.HF_JK_HOST | _abi.HF_JK_FP32_BOYS | _abi.HF_JK_DF64


def test_header_is_plain_c99_and_a_c_program_links(lib, tmp_path):
    """include/hf.h is a C interface: a C99 program (tests/c_abi_example.c)
    compiles against it without warnings, links to libhf.so and runs; with
    no GPU it stops at hf_ctx_create with HF_ERR_CUDA."""
    import shutil
    import subprocess
    import torch
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("no C compiler")
    libdir = os.path.join(ROOT, "paper_1303_4916_gb300")
    exe = str(tmp_path / "c_abi_example")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_example.c"), "-L", libdir, "-lhf", f"-Wl,-rpath,{libdir}",
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "tau 1e-12 max_iter 128" in out.stdout and "odd electron count" in out.stdout
    if not torch.cuda.is_available():
        assert "ctx -7" in out.stdout


def test_product_path_fails_loudly_without_the_library(tmp_path):
    """With libhf.so absent the package raises ImportError on first use;
    there is no CPU fallback to take over."""
    import subprocess
    import sys
    code = (
        "import paper_1303_4916_gb300._abi as a\n"
        f"a.load.__defaults__ = ({str(tmp_path / 'libhf.so')!r},)\n"
        "import paper_1303_4916_gb300 as hf\n"
        "try:\n"
        "    hf.jk_opts()\n"
        "except ImportError as e:\n"
        "    print('ImportError:', e)\n"
        "else:\n"
        "    print('no error')\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert "ImportError: libhf.so not built" in out.stdout, out.stdout + out.stderr
