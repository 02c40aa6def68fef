"""Host-side checks of the C-ABI library (no GPU compute): it loads, it
exports every entry point include/cq.h declares, the binding's names match,
and without a GPU it refuses to create a context instead of falling back."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cq.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cq_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2506_10092_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ["cq_ctx_create", "cq_column_create_rle", "cq_column_create_dict", "cq_column_create_index",
                 "cq_column_create_bitpacked", "cq_column_create_plain", "cq_table_bind", "cq_query_run",
                 "cq_result_fetch", "cq_align_segments", "cq_batch_run", "cq_server_create"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_c_names(libpath):
    from paper_2506_10092_gb300 import cq
    assert set(cq._SIGS) == set(declared())
    for n in declared():
        if n != "cq_last_error" and n not in ("cq_result_column_kind", "cq_column_encoding", "cq_table_num_rows",
                                              "cq_result_destroy", "cq_column_destroy", "cq_table_destroy",
                                              "cq_ctx_destroy", "cq_server_destroy"):
            assert hasattr(cq, n), n


def test_no_cpu_fallback_without_a_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_10092_gb300 import cq
    with pytest.raises(cq.CQError) as e:
        cq.cq_ctx_create(0)
    assert e.value.status == cq.CQ_ERR_CUDA


def test_oracle_is_not_reachable_from_the_product_path():
    """Nothing under the package imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2506_10092_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(import\s+oracle|from\s+oracle|liboracle|cq_oracle)", text), f


def test_every_exported_definition_is_declared():
    """No entry point is defined in the sources without a declaration in the
    public header (and so without its documentation)."""
    import glob
    src = ""
    for f in glob.glob(os.path.join(ROOT, "paper_2506_10092_gb300", "csrc", "*.cu")):
        src += open(f).read()
    defined = set(re.findall(r'extern "C"[^(]*?\b(cq_[a-z0-9_]+)\s*\(', src))
    assert defined and defined <= set(declared()), sorted(defined - set(declared()))


def test_generator_library_exports_its_header(libpath):
    gen_h = os.path.join(ROOT, "include", "cq_gen.h")
    names = sorted(set(re.findall(r"\b(cqgen_[a-z0-9_]+)\s*\(", re.sub(r"/\*.*?\*/", "", open(gen_h).read(),
                                                                         flags=re.S))))
    assert names == ["cqgen_hash_fields", "cqgen_nested_codes4"]
    lib = ctypes.CDLL(os.path.join(os.path.dirname(libpath), "libcqgen.so"))
    assert all(hasattr(lib, n) for n in names)


def test_specialised_row_kernel_compiles_without_a_gpu(libpath):
    """The run-time compiler builds the shape-specialised row kernel from the
    library's embedded device headers: eight check shapes that between them
    use every encoding, predicate kind, clause form, key mapping, aggregate
    layout and group table (shared hash table, run lines, global hash table,
    single group, dense table), with and without the warp pre-reduction and
    the serial walk of sorted data."""
    from paper_2506_10092_gb300 import cq
    for variant in range(8):
        secs = cq.cq_jit_check(variant)
        assert 0 < secs < 120
    with pytest.raises(cq.CQError) as e:
        cq.cq_jit_check(8)
    assert e.value.status == cq.CQ_ERR_INVALID_ARG
