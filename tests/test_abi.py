"""The C ABI without a GPU: the library loads, exports every function that
include/*.h declares, the ctypes structures match the C layout, and argument
validation answers before any device work."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1410_1914_gb300 import _lib, build
    build.build_cuda()
    return _lib.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(cl_\w+)\s*\(", text, flags=re.M):
            if not text[m.start():m.end()].lstrip().startswith("typedef"):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("cl_lbm_create", "cl_lbm_set_structure", "cl_lbm_solve", "cl_lbm_effective_diffusivity",
                     "cl_lbm_reaction_rate", "cl_lbm_destroy"):
        assert required in names


def declared_arity():
    """name -> number of parameters, from the prototypes in include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(cl_\w+)\s*\(([^;]*?)\)\s*;", text, flags=re.M):
            if m.group(0).lstrip().startswith("typedef"):
                continue
            args = m.group(2).strip()
            out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def _bindings():
    from paper_1410_1914_gb300 import _lib, warmstart
    sigs = {n: len(a) for n, (_, a) in _lib.SIGNATURES.items()}
    sigs.update({n: len(a) for n, (_, a) in warmstart._SIGS.items()})
    return sigs


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the bindings mirror every declared function, with the same arity
    sigs = _bindings()
    assert set(declared_functions()) <= set(sigs), set(declared_functions()) - set(sigs)
    arity = declared_arity()
    assert set(arity) == set(declared_functions())
    bad = {n: (k, sigs[n]) for n, k in arity.items() if sigs[n] != k}
    assert not bad, bad


def test_struct_layouts_match_c(tmp_path):
    from paper_1410_1914_gb300 import _lib
    structs = {"cl_params": _lib.cl_params, "cl_structure_info": _lib.cl_structure_info,
               "cl_solve_info": _lib.cl_solve_info, "cl_coupled_params": _lib.cl_coupled_params,
               "cl_coupled_info": _lib.cl_coupled_info, "cl_steady_info": _lib.cl_steady_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cl_lbm.h"', '#include "cl_nn.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} sizeof %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname} {f} %zu\\n", offsetof({sname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for ln in out:
        if not ln:
            continue
        sname, field, val = ln.split()
        cls = structs[sname]
        if field == "sizeof":
            assert ctypes.sizeof(cls) == int(val), sname
        else:
            assert getattr(cls, field).offset == int(val), (sname, field)


def test_defaults_and_strings(lib):
    from paper_1410_1914_gb300 import _lib
    p = _lib.cl_params_default()
    assert p.tau_ref == 1.0 and p.c_in == 1.0 and p.c_out == 0.0 and p.check_every == 1000
    assert p.storage == _lib.CL_STORE_FP32 and p.max_steps == 10_000_000
    assert _lib.status_str(_lib.CL_ERR_NO_PATH) == "CL_ERR_NO_PATH"
    assert "D3Q7" in _lib.version()


@pytest.mark.parametrize("field,value", [("nx", 0), ("tau_ref", 0.5), ("check_every", 3), ("bc_in", 7),
                                         ("storage", 9), ("dx_m", -1.0), ("k_ms", -1.0)])
def test_create_rejects_bad_parameters_before_device_work(lib, field, value):
    from paper_1410_1914_gb300 import _lib
    p = _lib.cl_params_default(nx=8, ny=8, nz=8)
    setattr(p, field, value)
    with pytest.raises(_lib.ClError) as e:
        _lib.cl_lbm_create(p)
    assert e.value.status == _lib.CL_ERR_ARG


def test_oversized_box_rejected(lib):
    from paper_1410_1914_gb300 import _lib
    p = _lib.cl_params_default(nx=2048, ny=2048, nz=1024)
    with pytest.raises(_lib.ClError) as e:
        _lib.cl_lbm_create(p)
    assert e.value.status == _lib.CL_ERR_ARG


def test_null_handle_calls(lib):
    from paper_1410_1914_gb300 import _lib
    info = _lib.cl_solve_info()
    assert lib.cl_lbm_solve(None, ctypes.byref(info)) == _lib.CL_ERR_ARG
    it = ctypes.c_int(-1)
    inner = ctypes.c_longlong(-1)
    assert lib.cl_lbm_solve_krylov(None, 1e-8, 10, 0, ctypes.byref(info), ctypes.byref(it)) == _lib.CL_ERR_ARG
    assert lib.cl_lbm_solve_krylov_dsa(None, 1e-8, 10, 0, ctypes.byref(info), ctypes.byref(it),
                                       ctypes.byref(inner)) == _lib.CL_ERR_ARG
    assert it.value == -1 and inner.value == -1  # outputs untouched on CL_ERR_ARG
    lib.cl_lbm_destroy(None)  # ignored


def test_property_formulas_match_the_oracle(lib):
    """Eq. 10, 11, 13 and the Tafel rate constant as host functions of the
    library equal the oracle's own evaluation (two independent statements of
    the printed formulas); no device work."""
    import math
    import oracle
    R, F = 8.314462618, 96485.33212
    for T in (300.0, 333.0, 353.0):
        assert lib.cl_henry_constant(T) == oracle.henry_constant(T)
        assert lib.cl_ionomer_o2_diffusivity(T) == oracle.ionomer_o2_diffusivity(T)
        assert lib.cl_ionomer_effective_diffusivity(T) == pytest.approx(
            oracle.ionomer_o2_diffusivity(T) * R * T / oracle.henry_constant(T), rel=1e-15)
    # Table 1 (Pt): i0m 0.01 A/m^2, alpha 0.61, phi_e 0.6 V, 333 K, c_ref 40.96 mol/m^3
    k = lib.cl_tafel_rate_constant(0.01, 0.61, 0.6, 333.0, 40.96)
    i_per_C = 0.01 * math.exp(0.61 * F * 0.6 / (R * 333.0)) * (R * 333.0 / oracle.henry_constant(333.0)) / 40.96
    assert k == pytest.approx(i_per_C / (4 * F), rel=1e-14)
    assert 1e-5 < k < 1e-4  # about 3.3e-5 m/s


def test_ionomer_o2_argument_checks(lib):
    from paper_1410_1914_gb300 import _lib as L
    p = L.cl_params_default(nx=4, ny=4, nz=4)
    p.ionomer_o2 = 1
    p.T_K = 280.0   # Eq. 13 is not positive below 283.7 K
    h = ctypes.c_void_p()
    assert lib.cl_lbm_create(ctypes.byref(h), ctypes.byref(p)) == L.CL_ERR_ARG
    p.T_K = 353.0
    p.carrier = L.CL_CARRIER_PROTON
    p.D_ionomer = 1.0
    assert lib.cl_lbm_create(ctypes.byref(h), ctypes.byref(p)) == L.CL_ERR_ARG


def test_noalloc_wrapper_checks_devices():
    """The allocation-free wrapper runs only on CUDA tensors of one device;
    the check answers on the host, before anything reaches the library."""
    import torch

    from paper_1410_1914_gb300 import _lib

    class _Fake:
        def __init__(self, kind, index):
            self.device = torch.device(kind, index) if kind == "cuda" else torch.device(kind)

    assert _lib._common_cuda_device(_Fake("cuda", 1), _Fake("cuda", 1)) == 1
    with pytest.raises(ValueError, match="different CUDA devices"):
        _lib._common_cuda_device(_Fake("cuda", 0), _Fake("cuda", 1))
    with pytest.raises(ValueError, match="CUDA tensors"):
        _lib._common_cuda_device(_Fake("cuda", 0), _Fake("cpu", None))
    cpu = torch.zeros((2, 2, 2), dtype=torch.uint8)
    with pytest.raises(ValueError):
        _lib.cl_active_mask_noalloc(cpu, torch.zeros_like(cpu))
