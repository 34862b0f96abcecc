"""Host-side checks of the C-ABI library that need no GPU: it loads, it
exports every function include/sem.h declares, and the host GLL set-up agrees
with the oracle (Sec. 2.2: GLL nodal basis)."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2501_13240_gb300 as sem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "sem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = sem.lib()
    names = header_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(sem.EXPORTS)


def test_version_and_error_text():
    assert "sm_103a" in sem.sem_version()
    assert isinstance(sem.lib().sem_last_error(), bytes)


@pytest.mark.parametrize("N", range(1, 11))
def test_library_gll_matches_oracle(N):
    xi, rho, D = sem.sem_gll(N)
    xo, ro, Do = oracle.gll(N)
    np.testing.assert_allclose(xi, xo, rtol=0, atol=2e-16)
    np.testing.assert_allclose(rho, ro, rtol=4e-16, atol=0)
    np.testing.assert_allclose(D, Do, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("N", [0, 11])
def test_library_gll_rejects_bad_order(N):
    with pytest.raises(sem.SemError) as ei:
        sem.sem_gll(N)
    assert ei.value.code == sem.SEM_ERR_INVALID_ARG


def test_write_ppm_host_only(tmp_path):
    """The PPM writer is host code: it runs without a GPU."""
    import paper_2501_13240_gb300 as sem
    img = np.zeros((2, 3, 4), dtype=np.uint8)
    img[0, :, 0] = 255   # bottom row red
    img[1, :, 2] = 255   # top row blue
    path = tmp_path / "x.ppm"
    sem.sem_write_ppm(str(path), img)
    data = path.read_bytes()
    head = b"P6\n3 2\n255\n"
    assert data[:len(head)] == head
    body = np.frombuffer(data[len(head):], dtype=np.uint8).reshape(2, 3, 3)
    assert (body[0, :, 2] == 255).all() and (body[1, :, 0] == 255).all()  # top row first in the file
    with pytest.raises(sem.SemError):
        sem.sem_write_ppm(str(tmp_path / "missing_dir" / "y.ppm"), img)


def test_every_entry_point_rejects_null_arguments():
    """Each C entry point, given NULL handles and pointers and zero sizes,
    returns SEM_ERR_INVALID_ARG with text naming the call, before touching a
    device; the destroy calls accept NULL as a no-op (like free)."""
    import ctypes
    L = sem.lib()
    destroys = {"sem_mesh_destroy", "sem_rbc_destroy", "sem_tadv_destroy", "sem_pmg_destroy", "sem_part_destroy"}
    ints = (ctypes.c_int, ctypes.c_uint, ctypes.c_int64)
    for name in sem.EXPORTS:
        if name in ("sem_last_error", "sem_version", "sem_pcg_noalloc_capacity", "sem_set_grid_wait_limit"):
            continue
        f = getattr(L, name)
        args = [0 if t in ints else 0.0 if t is ctypes.c_double else
                t() if isinstance(t, type) and issubclass(t, ctypes._CFuncPtr) else None  # NULL callback
                for t in f.argtypes]
        rc = f(*args)
        if name in destroys:
            assert rc == 0, name
        else:
            assert rc == -1, (name, rc)
            msg = L.sem_last_error().decode()
            assert msg.split(":")[0] in (name, "sem_partition"), (name, msg)


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the behaviour without a GPU")
def test_device_work_fails_loudly_without_a_gpu():
    """No CPU fallback: with no GPU the first call that needs one (building a
    mesh) returns SEM_ERR_CUDA with CUDA's message and hands out no mesh."""
    import ctypes
    d = sem.box_desc((2, 2, 2), 3)
    h = ctypes.c_void_p()
    rc = sem.lib().sem_mesh_create_box(ctypes.byref(d), None, ctypes.byref(h))
    assert rc == -2 and h.value is None
    assert "cuda" in sem.lib().sem_last_error().decode().lower()


def test_binding_refuses_host_tensors_for_device_arguments():
    """Device arguments must be contiguous CUDA tensors of the stated dtype
    and size: a host tensor is refused before any call into the library (the
    binding never computes on the CPU)."""
    import torch
    with pytest.raises(TypeError, match="CUDA tensor"):
        sem._ptr(torch.zeros(8, dtype=torch.float64), torch.float64, 8, "u")
    with pytest.raises(TypeError, match="CUDA tensor"):
        sem._ptr(np.zeros(8), torch.float64, 8, "u")


def test_readme_example_uses_existing_calls_and_keywords():
    """The README's Python example names only functions and keyword
    arguments the binding has (guards the documentation against drift)."""
    import ast
    import inspect
    txt = open(os.path.join(ROOT, "README.md")).read()
    code = txt.split("```python\n", 1)[1].split("```", 1)[0]
    tree = ast.parse(code)
    seen = 0
    for node in ast.walk(tree):
        if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name) and node.value.id == "sem":
            assert hasattr(sem, node.attr), node.attr
            seen += 1
        if isinstance(node, ast.Call) and isinstance(node.func, ast.Attribute) and \
                isinstance(node.func.value, ast.Name) and node.func.value.id == "sem":
            params = inspect.signature(getattr(sem, node.func.attr)).parameters
            for kw in node.keywords:
                assert kw.arg in params, (node.func.attr, kw.arg)
            assert len(node.args) <= len(params), node.func.attr
    assert seen >= 10


STRUCTS = ("sem_box_desc", "sem_mesh_info", "sem_solver_opts", "sem_solve_stats", "sem_pmg_opts", "sem_rbc_params",
           "sem_step_stats", "sem_rbc_view", "sem_tadv_params", "sem_slice_desc", "sem_scene_desc")


def test_binding_structs_match_the_c_header(tmp_path):
    """Every struct the binding passes by pointer has the size and field
    offsets the C compiler gives include/sem.h (a layout mismatch would
    corrupt arguments silently)."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sem.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(sem, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    c = {}
    for ln in out:
        if ln.strip():
            parts = ln.split()
            c[(parts[0], parts[1])] = int(parts[2])
    for name in STRUCTS:
        cls = getattr(sem, name)
        assert ctypes.sizeof(cls) == c[(name, "size")], name
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == c[(name, fname)], (name, fname)


def test_binding_signatures_match_the_c_prototypes():
    """Each function's ctypes argument list has the prototype's arity, and
    each argument the prototype's kind: pointer, int, unsigned, int64,
    size_t, double or one of the two callback types."""
    import ctypes
    txt = open(os.path.join(ROOT, "include", "sem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = dict((m.group(1), m.group(2)) for m in re.finditer(r"\b(sem_\w+)\s*\(([^)]*)\)\s*;", txt))
    L = sem.lib()
    scalar = {"int": ctypes.c_int, "double": ctypes.c_double, "int64_t": ctypes.c_int64, "size_t": ctypes.c_size_t,
              "unsigned": ctypes.c_uint, "sem_exchange_fn": sem.EXCHANGE_FN, "sem_allreduce_fn": sem.ALLREDUCE_FN}
    for name in sem.EXPORTS:
        params = [p.strip() for p in protos[name].split(",") if p.strip() and p.strip() != "void"]
        args = getattr(L, name).argtypes
        assert len(args) == len(params), (name, len(args), len(params))
        for p, a in zip(params, args):
            if "*" in p or "[" in p:
                assert a in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(a, ctypes._Pointer), (name, p, a)
            else:
                base = p.replace("const", "").split()[0]
                assert a is scalar[base] or (a is ctypes.c_int and base == "int"), (name, p, a)
