"""The C ABI without a GPU: the library loads, exports what include/admm.h
declares, and its host logic (partitioner, launch plan, argument checks)
behaves."""

import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT, gpu_available
from oracle import admm_fp64 as A

HEADER = os.path.join(ROOT, "include", "admm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(admm_[a-z_]+)\s*\(", text)))


def test_library_loads_and_exports_every_declared_symbol(cuda_lib):
    names = declared_functions()
    assert "admm_setup" in names and "admm_iterate" in names and "admm_solve" in names
    for name in names:
        assert hasattr(cuda_lib, name), name
    # and nothing that the binding expects is missing from the header
    from paper_1811_05571_gb300 import _binding
    assert set(_binding.SIGNATURES) == set(names)


def test_abi_version_and_strerror(cuda_lib):
    import paper_1811_05571_gb300 as P
    assert P.admm_abi_version() == P.ABI_VERSION == 5
    for code in range(0, 9):
        assert P.admm_strerror(code)
    assert P.admm_strerror(99) == "unknown status"


@pytest.mark.parametrize("total,parts", [(10, 3), (1440, 8), (32768, 8), (101, 4), (7, 7), (5, 1)])
def test_partition_matches_oracle_partitioner(cuda_lib, total, parts):
    import paper_1811_05571_gb300 as P
    off = P.admm_partition(total, parts)
    want = [a for a, _ in A.balanced_blocks(total, parts)] + [total]
    assert off == want


def test_partition_rejects_bad_arguments(cuda_lib):
    import paper_1811_05571_gb300 as P
    with pytest.raises(P.AdmmError):
        P.admm_partition(3, 4)
    with pytest.raises(P.AdmmError):
        P.admm_partition(3, 0)


PLAN_CASES = [(256, 4096, 4, 1), (1440, 32768, 8, 1), (1440, 32768, 1, 8), (1440, 32768, 4, 4),
              (100, 1000, 3, 3), (37, 517, 3, 5), (300, 3001, 7, 2), (12, 32, 1, 2),
              (2048, 16384, 8, 1), (8192, 131072, 16, 1), (16, 64, 4, 4), (96, 2048, 2, 16),
              (300, 3003, 3, 4), (200, 6001, 5, 4), (64, 20000, 1, 200)]


@pytest.mark.parametrize("m,n,M,N", PLAN_CASES)
def test_plan_slabs_cover_columns_and_fit_limits(cuda_lib, m, n, M, N):
    import paper_1811_05571_gb300 as P
    plan, slabs = P.admm_plan(m, n, M, N, num_sms=152, smem_limit=232448)
    ld = plan["ld"]
    assert ld >= n and ld % 32 == 0
    assert len(slabs) == plan["ctas"] <= 152
    beg = np.array([s[0] for s in slabs]); end = np.array([s[1] for s in slabs])
    own0 = np.array([s[2] for s in slabs]); own1 = np.array([s[3] for s in slabs])
    assert np.all(beg % 2 == 0) and np.all(end % 2 == 0) and np.all(end > beg)   # TMA x aligned
    assert beg[0] == 0 and end[-1] == ld
    # consecutive slabs abut or share the one pair holding an odd block boundary
    assert np.all((beg[1:] == end[:-1]) | (beg[1:] == end[:-1] - 2))
    assert (end - beg).max() == plan["slab_cols"]
    # every column (padding included) is owned by exactly one CTA, inside its slab
    assert np.all(own0 >= beg) and np.all(own1 <= end) and np.all(own1 > own0)
    assert own0[0] == 0 and own1[-1] == ld and np.all(own0[1:] == own1[:-1])
    assert np.all(own0 - beg <= 1) and np.all(end - own1 <= 1)
    col_off = [a for a, _ in A.balanced_blocks(n, N)] + [n]
    if N <= plan["ctas"]:
        assert plan["max_blocks_per_slab"] == 1
        # owned columns of a CTA never cross a column-block boundary
        for o0, o1 in zip(own0, own1):
            j = np.searchsorted(col_off, o0, side="right") - 1
            hi = col_off[j + 1] if j + 1 < N else ld
            assert o1 <= hi
        # slab widths are balanced within a column block
        for j in range(N):
            lo, hi = col_off[j], (col_off[j + 1] if j + 1 < N else ld)
            w = [e - b for b, e, o0, o1 in slabs if o0 >= lo and o1 <= hi]
            assert w and max(w) - min(w) <= 2
    assert plan["box_cols"] % 2 == 0 and plan["box_cols"] <= 256
    assert plan["box_cols"] * plan["boxes_per_row"] >= plan["slab_cols"]
    assert plan["groups"] in (1, 2)
    assert plan["slab_cols"] // 2 <= 32 * plan["chunks"] * plan["groups"]
    assert (plan["groups"] == 2) == (plan["slab_cols"] // 2 > 256)
    assert plan["rows_per_stage"] % 8 == 0 and 8 <= plan["rows_per_stage"] <= 64
    assert 2 <= plan["stages"] <= 8
    assert plan["smem_bytes"] <= 232448
    assert 1 <= plan["max_blocks_per_slab"] <= 4


def test_plan_rejects_too_narrow_column_blocks(cuda_lib):
    import paper_1811_05571_gb300 as P
    with pytest.raises(P.AdmmError) as e:
        P.admm_plan(8, 64, 1, 16, num_sms=1, smem_limit=232448)
    assert e.value.status == P.ADMM_EUNSUPPORTED


@pytest.mark.parametrize("kw,code", [
    (dict(m=0), 1), (dict(n=0), 1), (dict(M=9), 1), (dict(N=300), 1), (dict(M=16, N=17), 1),
    (dict(lam=-1.0), 1), (dict(lam=float("nan")), 1), (dict(rho=0.0), 1), (dict(rho=float("inf")), 1),
    (dict(dtype=7), 1),
])
def test_setup_argument_checks_need_no_gpu(cuda_lib, kw, code):
    """Invalid arguments are rejected on the host before any CUDA call."""
    import paper_1811_05571_gb300 as P
    args = dict(m=8, n=64, M=2, N=1, lam=0.1, rho=1.0, dtype=P.ADMM_C64)
    args.update(kw)
    H = np.zeros((max(args["m"], 1), max(args["n"], 1)), np.complex64)
    g = np.zeros(max(args["m"], 1), np.complex64)
    with pytest.raises(P.AdmmError) as e:
        P.admm_setup(H, g, args["m"], args["n"], args["M"], args["N"], args["lam"], args["rho"],
                     args["dtype"])
    assert e.value.status == code


def test_form_constants_match_the_header(cuda_lib):
    import paper_1811_05571_gb300 as P
    found = dict(re.findall(r"#define (ADMM_FORM_[A-Z]+)\s+(\d+)", open(HEADER).read()))
    assert {k: int(v) for k, v in found.items()} == {
        "ADMM_FORM_LEMMA": P.ADMM_FORM_LEMMA, "ADMM_FORM_DIRECT": P.ADMM_FORM_DIRECT,
        "ADMM_FORM_AUTO": P.ADMM_FORM_AUTO}


@pytest.mark.parametrize("form,n,N,code", [
    (3, 64, 1, 1), (-1, 64, 1, 1),
    (1, 12289, 1, 7), (1, 2 * 12288 + 1, 2, 7),   # a column block wider than 12288 columns
])
def test_setup_form_checks_need_no_gpu(cuda_lib, form, n, N, code):
    """An unknown factor form, and a direct form whose column blocks are too
    wide for it, are rejected on the host before any CUDA call."""
    import paper_1811_05571_gb300 as P
    H = np.zeros((8, 1), np.complex64)   # never read: the checks come first
    g = np.zeros(8, np.complex64)
    with pytest.raises(P.AdmmError) as e:
        P.admm_setup_form(H, g, 8, n, 1, N, 0.1, 1.0, P.ADMM_C64, form)
    assert e.value.status == code


def test_null_pointers_rejected(cuda_lib):
    import paper_1811_05571_gb300 as P
    h = ctypes.c_void_p()
    assert cuda_lib.admm_setup(ctypes.byref(h), None, None, 4, 8, 1, 1, 0.1, 1.0, 0, None) == P.ADMM_EINVAL
    assert cuda_lib.admm_setup(None, None, None, 4, 8, 1, 1, 0.1, 1.0, 0, None) == P.ADMM_EINVAL
    assert cuda_lib.admm_iterate(None, 1, None) == P.ADMM_EINVAL
    assert cuda_lib.admm_get_info(None, None) == P.ADMM_EINVAL
    cuda_lib.admm_destroy(None)


@pytest.mark.skipif(gpu_available(), reason="checks the no-GPU error path")
def test_setup_without_gpu_reports_cuda_error(cuda_lib):
    import paper_1811_05571_gb300 as P
    H = np.zeros((4, 64), np.complex64)
    g = np.zeros(4, np.complex64)
    with pytest.raises(P.AdmmError) as e:
        P.admm_setup(H, g, 4, 64, 2, 1, 0.1, 1.0)
    assert e.value.status == P.ADMM_ECUDA


def test_comm_elements_follow_table1_and_table3(cuda_lib):
    """The host-side communication counts match the oracle's Table I formulas
    exactly and reproduce the printed Table III counts (M = 4, N = 3,
    N_m = 2160, N_p = 22500) where they follow from Table I."""
    import paper_1811_05571_gb300 as P
    for m, n in ((2160, 22500), (1440, 32768), (37, 517)):
        for M in (1, 2, 4, 7):
            for N in (1, 3, 8):
                assert P.admm_comm_elements(m, n, M, N) == A.comm_elements(M, N, m, n)
    c = P.admm_comm_elements(2160, 22500, 4, 3)
    assert c["consensus"] == 45000 and c["sectioning"] == 6480 and c["cs"] == 16620
    for bad in ((0, 5, 1, 1), (5, 0, 1, 1), (5, 5, 0, 1), (5, 5, 1, 0)):
        with pytest.raises(P.AdmmError):
            P.admm_comm_elements(*bad)


@pytest.mark.parametrize("kw,code", [
    (dict(batch=0), 1), (dict(lam_bad=True), 1), (dict(m=10), 7), (dict(M=3, m=20), 7),
])
def test_batch_setup_argument_checks_need_no_gpu(cuda_lib, kw, code):
    """The batched solver rejects bad sizes and block starts off the 4-element
    grid of its FP16 tensor maps on the host, before any CUDA call."""
    import paper_1811_05571_gb300 as P
    args = dict(m=16, n=64, M=2, N=1, batch=2)
    args.update({k: v for k, v in kw.items() if k != "lam_bad"})
    H = np.zeros((args["m"], args["n"]), np.complex64)
    lam = [0.1] * max(args["batch"], 1)
    if kw.get("lam_bad"):
        lam[0] = float("nan")
    with pytest.raises(P.AdmmError) as e:
        P.admm_batch_setup(H, args["m"], args["n"], args["M"], args["N"], args["batch"], lam, 1.0,
                           P.ADMM_C64)
    assert e.value.status == code
