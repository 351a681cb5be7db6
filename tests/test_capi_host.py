"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every symbol include/lasp.h declares, and rejects bad arguments before any
device work."""
import ctypes as ct
import math
import os
import re

import numpy as np
import pytest

import lasp_synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lasp():
    from paper_2512_24840_gb300 import lasp as L
    L.load(build=True)
    return L


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"\b(lasp_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lasp):
    lib = lasp.load()
    declared = _declared()
    assert declared >= set(lasp.EXPORTS)
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_strerror_and_defaults(lasp):
    assert lasp.strerror(0) == "ok"
    assert "invalid" in lasp.strerror(-1)
    o = lasp.default_opts()
    assert abs(o.lr - 0.1) < 1e-7 and o.window == 50 and o.max_steps == 5000
    assert o.legendre_deg == 6 and abs(o.quantile - 0.5) < 1e-7 and abs(o.tol - 1e-5) < 1e-12


def _desc(lasp, g, pad=None, K=None, exps=None):
    exps = S.EXPS if exps is None else exps
    return lasp.InterpDesc(len(exps) if K is None else K, g.n_pix, g.pad if pad is None else pad,
                           g.dln, exps.ctypes.data, (ct.c_double * 3)(*S.BASIS_LO),
                           (ct.c_double * 3)(*S.BASIS_HI), (ct.c_double * 5)(*S.BOX_LO),
                           (ct.c_double * 5)(*S.BOX_HI))


def test_init_validation(lasp):
    lib = lasp.load()
    g = S.SMALL
    C = np.zeros((26, g.n_model), dtype=np.float32)
    h = ct.c_void_p()
    exps = np.ascontiguousarray(S.EXPS)
    # pad smaller than the widest kernel of the box (Eq. 5)
    d = _desc(lasp, g, pad=g.pad - 1, exps=exps)
    assert lib.lasp_init_interp(ct.byref(d), C.ctypes.data, ct.byref(h)) == lasp.EGRID
    d = _desc(lasp, g, K=0, exps=exps)
    assert lib.lasp_init_interp(ct.byref(d), C.ctypes.data, ct.byref(h)) == lasp.EINVAL
    bad = exps.copy()
    bad[3, 0] = -1
    d = _desc(lasp, g, exps=bad)
    assert lib.lasp_init_interp(ct.byref(d), C.ctypes.data, ct.byref(h)) == lasp.EINVAL
    assert lib.lasp_init_interp(None, C.ctypes.data, ct.byref(h)) == lasp.EINVAL
    # the largest accepted sizes: 8192 model pixels (n_pix + 2 pad), a margin of 47 pixels
    big = S.Grid("over", 8192 - 2 * S.DESI.pad + 1, 3600.0, S.DESI.dln)
    assert big.n_model == 8193
    Cb = np.zeros((26, big.n_model), dtype=np.float32)
    d = _desc(lasp, big, exps=exps)
    assert lib.lasp_init_interp(ct.byref(d), Cb.ctypes.data, ct.byref(h)) == lasp.EINVAL
    d = _desc(lasp, g, pad=48, exps=exps)
    Cp = np.zeros((26, g.n_pix + 96), dtype=np.float32)
    assert lib.lasp_init_interp(ct.byref(d), Cp.ctypes.data, ct.byref(h)) == lasp.EINVAL
    assert not h.value


def test_no_device_is_reported(lasp):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = lasp.load()
    g = S.SMALL
    C = np.zeros((26, g.n_model), dtype=np.float32)
    exps = np.ascontiguousarray(S.EXPS)
    d = _desc(lasp, g, exps=exps)
    h = ct.c_void_p()
    assert lib.lasp_init_interp(ct.byref(d), C.ctypes.data, ct.byref(h)) == lasp.ENODEV


def test_null_handle_calls_fail_cleanly(lasp):
    lib = lasp.load()
    o = lasp.default_opts()
    b = lasp.Batch(4, 1024, None, None, None, None)
    r = lasp.Result()
    assert lib.lasp_fit_batch(None, ct.byref(b), ct.byref(o), ct.byref(r), None) == lasp.EINVAL
    assert lib.lasp_forward(None, 1, None, None, 6, None, None) == lasp.EINVAL
    assert lib.lasp_backward(None, 1, None, None, 6, None, None, None, None) == lasp.EINVAL
    assert lib.lasp_interp_eval(None, 1, None, None, 0, None) == lasp.EINVAL
    lib.lasp_free_interp(None)
    # slot pools and the native server: null handles and bad counts
    P = ct.c_void_p
    lib.lasp_slots_step.argtypes = [P, ct.c_int, P]
    lib.lasp_slots_step_running.argtypes = [P, ct.c_int, ct.c_int, P]
    lib.lasp_slots_admit.argtypes = [P, ct.c_int, P, P, P, P, P, P]
    lib.lasp_slots_fetch.argtypes = [P, P, P, P, P, P, P]
    assert lib.lasp_slots_step(None, 25, None) == lasp.EINVAL
    assert lib.lasp_slots_step_running(None, 25, 10, None) == lasp.EINVAL
    assert lib.lasp_slots_admit(None, 1, None, None, None, None, None, None) == lasp.EINVAL
    assert lib.lasp_slots_fetch(None, None, None, None, None, None, None) == lasp.EINVAL
    lib.lasp_slots_free(None)
    n = ct.c_int(-1)
    lib.lasp_server_tick.argtypes = [P, ct.POINTER(ct.c_int)]
    assert lib.lasp_server_tick(None, ct.byref(n)) == lasp.EINVAL and n.value == 0
    lib.lasp_server_pending.argtypes = [P, ct.POINTER(ct.c_int64)]
    assert lib.lasp_server_pending(None, ct.byref(ct.c_int64())) == lasp.EINVAL
    taken = ct.c_int(-1)
    assert lib.lasp_server_submit_n(None, 0, 1, None, None, None, None, None,
                                    ct.byref(taken)) == lasp.EINVAL and taken.value == 0
    assert lib.lasp_server_submit_n(None, 0, 1, None, None, None, None, None, None) == lasp.EINVAL


def test_header_is_plain_c(tmp_path):
    """include/lasp.h is a C header: a C99 translation unit using it compiles
    cleanly (-Wall -Wextra -pedantic -Werror)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "use_lasp.c"
    src.write_text('#include "lasp.h"\n'
                   "int main(void) {\n"
                   "    lasp_fit_opts o;\n"
                   "    lasp_default_opts(&o);\n"
                   "    return lasp_version() > 0 && o.window == 50 ? 0 : 1;\n"
                   "}\n")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-c",
                        f"-I{inc}", str(src), "-o", str(tmp_path / "use_lasp.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_binding_checks_tensor_shapes_before_any_call(lasp):
    """The binding checks each tensor's dtype and shape before its pointer
    reaches the library (which sizes every buffer from N and the grid), then
    that it is a contiguous CUDA tensor: host tensors never reach a kernel."""
    torch = pytest.importorskip("torch")
    ip = object.__new__(lasp.Interp)
    ip._h, ip.n_pix, ip.n_model = None, 16, 56
    f = lambda *shape: torch.zeros(shape, dtype=torch.float32)
    with pytest.raises(ValueError, match="theta"):
        ip.forward(f(3, 4), f(3, 7))
    with pytest.raises(ValueError, match="b"):
        ip.forward(f(3, 5), f(2, 7))
    with pytest.raises(ValueError, match="gmodel"):
        ip.backward(f(3, 5), f(3, 7), f(3, 15))
    with pytest.raises(ValueError, match="theta"):
        ip.interp_eval(f(3, 5, 1))
    with pytest.raises(TypeError, match="b"):
        ip.forward(f(3, 5), torch.zeros((3, 7), dtype=torch.float64))
    # right dtypes and shapes, but host tensors
    with pytest.raises(TypeError, match="CUDA"):
        ip.backward(f(3, 5), f(3, 7), f(3, 16))
    with pytest.raises(TypeError, match="CUDA"):
        ip.forward(f(0, 5), f(0, 7))


def test_every_accepted_grid_can_launch(tmp_path):
    """tests/limits_host.cu, built as host code and run here: over every grid
    lasp_init_interp accepts, the fit kernels' blocks cover the model grid and
    every kernel's shared memory fits a CTA (no device needed)."""
    import shutil
    import subprocess
    nvcc = next((c for c in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")) if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("no nvcc")
    exe = tmp_path / "limits_host"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=compute_103a", "-O1", "-std=c++17",
                        f"-I{os.path.join(ROOT, 'include')}",
                        f"-I{os.path.join(ROOT, 'paper_2512_24840_gb300', 'csrc')}",
                        os.path.join(ROOT, "tests", "limits_host.cu"), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout


def _pw_desc(lasp, g, Ks, pad=None, n_pix=None, tb=(4000.0, 4550.0, 7000.0, 9000.0)):
    exps = np.ascontiguousarray(np.concatenate([S.EXPS[:k] for k in Ks]), dtype=np.int8) \
        if sum(Ks) <= 3 * len(S.EXPS) else np.zeros((sum(Ks), 3), np.int8)
    d = lasp.PiecewiseDesc()
    d.n_reg = len(Ks)
    for r, k in enumerate(Ks[:3]):
        d.K[r] = k
    d.n_pix = g.n_pix if n_pix is None else n_pix
    d.pad = g.pad if pad is None else pad
    d.dln = g.dln
    d.exps = exps.ctypes.data
    lo = [math.log10(3000.0), 0.5, -2.5]
    for r in range(3):
        for k in range(3):
            d.basis_lo[r][k] = lo[k] + 0.1 * r
            d.basis_hi[r][k] = lo[k] + 1.0 + 0.1 * r
    d.teff_blend = (ct.c_double * 4)(*tb)
    d.box_lo = (ct.c_double * 5)(*S.BOX_LO)
    d.box_hi = (ct.c_double * 5)(*S.BOX_HI)
    return d, exps


def test_piecewise_init_validation(lasp):
    """lasp_init_interp_piecewise rejects bad descriptors before any device
    work: regime count outside 1..3, a regime without terms, more than 96 rows,
    blend bounds not increasing, a margin above 47 or a model grid above 8192
    pixels (LASP_EINVAL), and a margin too small for the box (LASP_EGRID)."""
    lib = lasp.load()
    lib.lasp_init_interp_piecewise.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
    g = S.SMALL
    h = ct.c_void_p()
    C = np.zeros((200, g.n_pix + 2 * 47 + 200), dtype=np.float32)

    def rc(*a, **k):
        d, exps = _pw_desc(lasp, g, *a, **k)
        return lib.lasp_init_interp_piecewise(ct.byref(d), C.ctypes.data, ct.byref(h))

    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        # the descriptor the cases below spoil one field of is itself valid:
        # without a device it gets as far as the device check
        assert rc([25, 26, 19]) == lasp.ENODEV
    d, _ = _pw_desc(lasp, g, [25, 26, 19])
    d.n_reg = 0
    assert lib.lasp_init_interp_piecewise(ct.byref(d), C.ctypes.data, ct.byref(h)) == lasp.EINVAL
    d.n_reg = 4
    assert lib.lasp_init_interp_piecewise(ct.byref(d), C.ctypes.data, ct.byref(h)) == lasp.EINVAL
    assert rc([25, 0, 19]) == lasp.EINVAL
    assert rc([40, 40, 20]) == lasp.EINVAL                       # 100 rows > 96
    assert rc([25, 26, 19], tb=(4000.0, 3900.0, 7000.0, 9000.0)) == lasp.EINVAL
    assert rc([25, 26, 19], pad=48) == lasp.EINVAL
    assert rc([25, 26, 19], n_pix=8192 - 2 * g.pad + 1) == lasp.EINVAL
    assert rc([25, 26, 19], pad=g.pad - 1) == lasp.EGRID
    assert lib.lasp_init_interp_piecewise(None, C.ctypes.data, ct.byref(h)) == lasp.EINVAL
    assert not h.value


def test_binding_structs_match_the_header(lasp, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    of the C struct in include/lasp.h (compiled by the host C compiler), and
    the numpy view of lasp_served matches too."""
    import shutil
    import subprocess
    from paper_2512_24840_gb300 import server
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"lasp_interp_desc": lasp.InterpDesc, "lasp_piecewise_desc": lasp.PiecewiseDesc,
               "lasp_batch": lasp.Batch, "lasp_fit_opts": lasp.FitOpts, "lasp_result": lasp.Result,
               "lasp_kernel_time": lasp.KernelTime, "lasp_served": server._Served}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "lasp.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            cname, field, v = line.split()
            c[(cname, field)] = int(v)
    for cname, cls in structs.items():
        assert ct.sizeof(cls) == c[(cname, "size")], cname
        for f in cls._fields_:
            assert getattr(cls, f[0]).offset == c[(cname, f[0])], (cname, f[0])
    dt = server._SERVED_DT
    assert dt.itemsize == c[("lasp_served", "size")]
    for name in dt.names:
        assert dt.fields[name][1] == c[("lasp_served", name)], name


def _prototypes():
    """name -> (return type, [parameter types]) of every lasp_* prototype in
    include/lasp.h, each parameter reduced to pointer / int / int64 / float /
    double (the opaque handle typedefs are pointers)."""
    txt = open(os.path.join(ROOT, "include", "lasp.h")).read()
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    txt = re.sub(r"^\s*#.*$", " ", txt, flags=re.M)           # preprocessor lines
    txt = re.sub(r"\s+", " ", txt)
    handles = {"lasp_interp", "lasp_slots", "lasp_server"}
    kinds = {"int": "int", "int32_t": "int", "uint32_t": "int", "int64_t": "int64", "float": "float",
             "double": "double"}
    protos = {}
    for chunk in re.split(r"[;{}]", txt):
        m = re.fullmatch(r"\s*([A-Za-z_][\w ]*?\**)\s*\b(lasp_\w+)\s*\(([^)]*)\)\s*", chunk)
        if not m or m.group(1).strip() in ("typedef", "struct"):
            continue
        ret, name, params = m.groups()
        ps = []
        for prm in [p.strip() for p in params.split(",")]:
            if prm in ("", "void"):
                continue
            words = prm.replace("*", " * ").split()
            if "*" in words:
                ps.append("pointer")
            else:
                base = [w for w in words[:-1] if w not in ("const", "unsigned")]
                ps.append("pointer" if base[-1] in handles else kinds[base[-1]])
        protos[name] = (ret.strip(), ps)
    return protos


def test_binding_signatures_match_the_header(lasp):
    """The argument lists the binding declares to ctypes have the header's
    arity and, parameter by parameter, its kind (pointer, int, int64, float,
    double)."""
    lib = lasp.load()
    protos = _prototypes()
    kind = {ct.c_void_p: "pointer", ct.c_char_p: "pointer", ct.c_int: "int", ct.c_int64: "int64",
            ct.c_float: "float", ct.c_double: "double"}
    checked = 0
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        if fn.argtypes is None:
            continue              # declared where it is used (slot pools, tests)
        got = [kind.get(a, "pointer" if hasattr(a, "contents") or a.__name__.startswith("LP_") else "?")
               for a in fn.argtypes]
        assert got == params, (name, got, params)
        checked += 1
    assert checked >= 20, checked
    assert protos["lasp_strerror"][0].endswith("*") and lib.lasp_strerror.restype is ct.c_char_p
