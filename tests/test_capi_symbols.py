"""The C-ABI library builds, loads without a GPU, and exports every entry point of include/sph.h."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1309_3783_gb300 import build
    return build.build()


def test_header_declares_the_interface():
    names = _declared()
    for want in ("sph_ctx_create", "sph_box_create", "sph_build", "sph_density", "sph_h_update", "sph_force",
                 "sph_step", "sph_get", "sph_server_tick"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sph_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_covers_the_header(lib_path):
    from paper_1309_3783_gb300 import sph
    lib = sph.load()
    assert set(sph.exported_symbols()) == set(_declared())
    p = sph.sph_params_default()      # host-only entry point: no GPU needed
    assert abs(p.gamma_kernel - 1.825742) < 1e-6 and p.n_ngb == 48 and p.leaf_max == 400
    assert abs(p.split_frac - 0.875) < 1e-7 and p.h_max_iter == 30
    assert lib is not None


def test_context_creation_fails_cleanly_without_a_device(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_1309_3783_gb300 import sph
    with pytest.raises(sph.SphError):
        sph.sph_ctx_create(device=0)


def _header_struct(name):
    """(field, C type) of `typedef struct name { ... } name;` in include/sph.h, in order."""
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, flags=re.S).group(1)
    return re.findall(r"\b(int32_t|int64_t|float|double|char)\s+(\w+)\s*(?:\[\d+\])?\s*;", body)


@pytest.mark.parametrize("name", ["sph_params", "sph_stats", "sph_profile_entry"])
def test_binding_structs_mirror_the_header(name):
    import ctypes as C
    from paper_1309_3783_gb300 import sph
    width = {"int32_t": 4, "int64_t": 8, "float": 4, "double": 8}
    want = _header_struct(name)
    got = getattr(sph, name)._fields_
    assert [f for _, f in want] == [f for f, _ in got]
    for (ctype, field), (_, pytype) in zip(want, got):
        if ctype != "char":
            assert C.sizeof(pytype) == width[ctype], field
        if ctype in ("float", "double"):
            assert pytype in (C.c_float, C.c_double), field


def test_parameter_defaults_of_the_options(lib_path):
    from paper_1309_3783_gb300 import sph
    p = sph.sph_params_default()
    assert p.graphs == 1 and p.h_gather == 1 and p.pair_cache == 0 and p.reuse == 0 and p.sort_merge == 0
    assert p.cluster_max == 32 and p.compensated == -1 and p.precision == 0
