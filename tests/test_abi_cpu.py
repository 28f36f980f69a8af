"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/neumann.h declares, validates arguments and plans the paper's
product counts."""

import os
import re

import pytest

from tests.conftest import ROOT

nm = pytest.importorskip("paper_2602_11843_gb300", reason="library not built")
from paper_2602_11843_gb300 import _capi as C  # noqa: E402

from oracle import counts as CT  # noqa: E402
from oracle import radix15 as R15
from oracle import radix_p5 as RP5  # noqa: E402


def test_exports_every_declared_symbol():
    import ctypes

    hdr = open(os.path.join(ROOT, "include", "neumann.h")).read()
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(neumann_\w+)\s*\(", hdr, re.M)
    assert len(names) >= 12
    lib = ctypes.CDLL(C.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("n,k,radix,dtype,flags", [
    (0, 81, 9, C.FP64, 0), (10, 0, 9, C.FP64, 0), (10, 80, 9, C.FP64, 0), (10, 100, 15, C.FP64, 0),
    (10, 12, 2, C.FP64, 0), (10, 7 * 9, 0, C.FP64, 0), (10, 81, 7, C.FP64, 0), (10, 81, 9, 9, 0),
    (10, 625, 24, C.FP64, 0), (10, 576, 25, C.FP64, 0), (10, 576, 23, C.FP64, 0),
])
def test_invalid_arguments(n, k, radix, dtype, flags):
    with pytest.raises(C.NeumannError) as e:
        C.neumann_plan_create(n, k, radix, dtype, flags)
    assert e.value.code == C.EINVAL


def test_fp16_plan_has_the_split_layout():
    """The split-FP16 plan has the BF16 plan's matrices plus its scaling records
    (max |x|, column-sum bound and exponent per output, column sums of the
    products' right operands): a few KB at this order."""
    h = C.neumann_plan_create(64, 81, 9, C.SPLIT_FP16, 0)
    hb = C.neumann_plan_create(64, 81, 9, C.SPLIT_BF16, 0)
    try:
        a, b = C.neumann_plan_info(h), C.neumann_plan_info(hb)
        assert 0 < a["workspace_bytes"] - b["workspace_bytes"] < 64 * 1024
        assert a["products_executed"] == b["products_executed"] == 8
    finally:
        C.neumann_plan_destroy(h)
        C.neumann_plan_destroy(hb)


def _info(n, k, radix, dtype=C.FP64, flags=0):
    h = C.neumann_plan_create(n, k, radix, dtype, flags)
    try:
        return C.neumann_plan_info(h)
    finally:
        C.neumann_plan_destroy(h)


@pytest.mark.parametrize("k,radix", [(81, 9), (729, 9), (6561, 9), (225, 15), (3375, 15), (125, 5), (625, 5),
                                     (27, 3), (128, 2), (1024, 2), (4096, 2), (24, 24), (576, 24),
                                     (13824, 24), (625, 25), (15625, 25)])
def test_product_counts_match_paper(k, radix):
    """products_formula = the paper's count (Table tab:results, Sec. 2.2 cost model,
    Sec. 6 binary); products_executed = formula - 2 (no product with S_1 = I, no unused power)."""
    info = _info(64, k, radix)
    formula = CT.binary_formula(k) if radix == 2 else CT.radix_formula(k, radix)
    assert info["products_formula"] == formula
    assert info["products_executed"] == formula - 2
    assert info["levels"] == [radix] * len(info["levels"])


def test_naive_and_exact_binary_counts():
    assert _info(32, 81, 1)["products_executed"] == 79
    assert _info(32, 81, 1)["products_formula"] == 80
    for k in (81, 100, 225, 729, 3375, 6561):
        L, ones = k.bit_length(), bin(k).count("1")
        assert _info(32, k, 2, flags=C.FLAG_EXACT_K)["products_executed"] == 2 * L + ones - 5


def test_auto_levels():
    info = _info(32, 2 * 3 * 5 * 9, 0)
    assert sorted(info["levels"]) == [2, 3, 5, 9]
    assert info["products_formula"] == 2 + 3 + 4 + 5


@pytest.mark.parametrize("k", [1, 2])
def test_trivial_k_has_no_products(k):
    for radix in (1, 2, 9):
        if radix == 9 and k == 2:
            continue
        assert _info(16, k, radix)["products_executed"] == 0


def test_workspace_layout_padded():
    info = _info(300, 81, 9, C.SPLIT_BF16)
    assert info["padded_n"] == 512
    assert info["workspace_bytes"] % 256 == 0 and info["workspace_bytes"] > 512 * 512 * 8


def test_library_radix15_coefficients_match_oracle():
    """The library refines the App. B values on the host in double precision;
    the oracle refines them in multi-precision. Same reading, same solution."""
    coef, err, s15, s16 = C.neumann_radix15_coefficients(0)
    ref = R15.flatten(R15.load_refined(float))
    assert max(abs(a - b) for a, b in zip(coef, ref)) < 1e-13
    assert err < 1e-14
    assert abs(s15 - 0.18520417118533553) < 1e-12 and abs(s16 - 0.4583601331249466) < 1e-12
    pcoef, perr, _, _ = C.neumann_radix15_coefficients(1)
    assert pcoef == R15.flatten(R15.printed(float))
    assert 2e-3 < perr < 4e-3


@pytest.mark.parametrize("m", RP5.RADICES)
def test_library_radix_p5_coefficients_match_oracle(m):
    """The library refines the published six-decimal circuit in double precision;
    the oracle refines it in multi-precision. Same start, same solution."""
    coef, err, spill = C.neumann_radix_p5_coefficients(m)
    ref = RP5.flatten(RP5.load_refined(m))
    assert max(abs(a - b) for a, b in zip(coef, ref)) < 1e-12
    assert err < 1e-13
    assert abs(spill - float(RP5.refined_metadata(m)["spill"])) < 1e-12
    for bad in (15, 23, 26):
        with pytest.raises(C.NeumannError) as e:
            C.neumann_radix_p5_coefficients(bad)
        assert e.value.code == C.EINVAL


@pytest.mark.parametrize("radix,k", [(24, 576), (25, 15625), (27, 729), (31, 961), (33, 1089)])
def test_five_product_levels_pass_count(radix, k):
    """A single five-product plan forms the fifth factors in the fourth product's
    epilogue, with the third power's share read from C (no element-wise pass);
    a grouped batch folds their parts into the third product's epilogue. Both
    launch only the split of A and the products."""
    levels = {576: 2, 15625: 3, 729: 2, 961: 2, 1089: 2}[k]
    h = C.neumann_plan_create(1024, k, radix, C.SPLIT_BF16, 0)
    try:
        i = C.neumann_plan_info(h)
    finally:
        C.neumann_plan_destroy(h)
    assert i["products_executed"] == 7 * levels - 2
    assert i["launches"] == i["products_executed"] + 1
    hb = C.neumann_plan_create_batched(64, 256, k, radix, C.SPLIT_BF16, 0)
    try:
        ib = C.neumann_plan_info(hb)
    finally:
        C.neumann_plan_destroy(hb)
    assert ib["products_executed"] == 7 * levels - 2
    assert ib["launches"] == ib["products_executed"] + 1


def test_batched_plan_and_empty_batch():
    h = C.neumann_plan_create_batched(4, 256, 81, 9, C.FP32, 0)
    try:
        C.neumann_eval_batched(h, [], [], [])  # empty batch is a no-op
        with pytest.raises(C.NeumannError):
            C.neumann_eval_batched(h, [300], [1], [2])  # n above max_n
    finally:
        C.neumann_plan_destroy(h)


def test_launch_configuration_defaults():
    """Before tuning: CTA pairs from padded order 4096, raster groups of 8, one
    pass of up to 2048 matrices for a grouped batch."""
    assert _info(4096, 81, 9, C.SPLIT_BF16)["tile_pair"] == 1
    assert _info(4000, 81, 9, C.SPLIT_FP16)["tile_pair"] == 1
    assert _info(3840, 81, 9, C.SPLIT_BF16)["tile_pair"] == 0
    assert _info(8192, 81, 9, C.SPLIT_BF16, C.FLAG_SINGLE_CTA)["tile_pair"] == 0
    i = _info(300, 81, 9, C.SPLIT_BF16)
    assert i["raster_group"] == 8 and i["tuned"] == 0 and i["batch_chunk"] == 0
    assert _info(4096, 81, 9, C.FP64)["tile_pair"] == 0
    h = C.neumann_plan_create_batched(3000, 256, 81, 9, C.SPLIT_BF16, 0)
    try:
        assert C.neumann_plan_info(h)["batch_chunk"] == 2048
    finally:
        C.neumann_plan_destroy(h)


def test_set_launch_host_only():
    """A hand-set launch configuration shows in the plan's info; out-of-range
    values and plans without tensor-core products are refused. No workspace is
    attached, so nothing touches a device."""
    h = C.neumann_plan_create(8192, 3375, 15, C.SPLIT_BF16, 0)
    h32 = C.neumann_plan_create(64, 81, 9, C.FP32, 0)
    hb = C.neumann_plan_create_batched(4, 64, 81, 9, C.SPLIT_BF16, 0)
    try:
        i = C.neumann_plan_info(h)
        assert (i["tile_pair"], i["raster_group"], i["tuned"]) == (1, 8, 0)
        C.neumann_plan_set_launch(h, 0, 4)
        i = C.neumann_plan_info(h)
        assert (i["tile_pair"], i["raster_group"], i["tuned"]) == (0, 4, 1)
        C.neumann_plan_set_launch(h, -1, 16)
        i = C.neumann_plan_info(h)
        assert (i["tile_pair"], i["raster_group"]) == (1, 16)
        for args in [(h, 2, 8), (h, 1, 0), (h, 1, 1 << 16), (h, -2, 8), (h32, 1, 8), (hb, 1, 8)]:
            with pytest.raises(C.NeumannError) as e:
                C.neumann_plan_set_launch(*args)
            assert e.value.code == C.EINVAL
    finally:
        for x in (h, h32, hb):
            C.neumann_plan_destroy(x)


def test_autotune_argument_errors():
    """Rejected before any device work."""
    h = C.neumann_plan_create(64, 81, 9, C.SPLIT_BF16, 0)
    hb = C.neumann_plan_create_batched(4, 64, 81, 9, C.SPLIT_BF16, 0)
    try:
        for args in [(h, 16, 64, 32, 64, 0), (hb, 16, 64, 32, 64, 3), (h, 16, 63, 32, 64, 3), (h, 0, 64, 32, 64, 3)]:
            with pytest.raises(C.NeumannError) as e:
                C.neumann_plan_autotune(*args)
            assert e.value.code == C.EINVAL
        for args in [(h, [64], [16], [32], 3), (hb, [65], [16], [32], 3), (hb, [64], [16], [32], 0),
                     (hb, [64] * 5, [16] * 5, [32] * 5, 3)]:
            with pytest.raises(C.NeumannError) as e:
                C.neumann_plan_autotune_batched(*args)
            assert e.value.code == C.EINVAL
    finally:
        C.neumann_plan_destroy(h)
        C.neumann_plan_destroy(hb)


def test_algorithmic_bytes_per_element():
    """The plan's byte count per matrix element grows with the work: more levels
    move more bytes, the products are most of them, and FP64 moves the most."""
    b9 = _info(512, 81, 9, C.SPLIT_BF16)
    b9x = _info(512, 729, 9, C.SPLIT_BF16)
    assert 0 < b9["product_bytes_per_element"] < b9["bytes_per_element"]
    assert b9x["bytes_per_element"] > b9["bytes_per_element"]
    # per product, between the bare operands (8 B of hi/lo pairs) and operands plus
    # four inputs and four outputs in every representation
    per = b9["product_bytes_per_element"] / b9["products_executed"]
    assert 8 < per < 8 + 4 * 8 + 4 * 20
    assert _info(512, 81, 9, C.FP64)["bytes_per_element"] > _info(512, 81, 9, C.FP32)["bytes_per_element"]


def test_eval_host_argument_errors():
    h = C.neumann_plan_create(64, 81, 9, C.SPLIT_BF16, 0)
    hb = C.neumann_plan_create_batched(4, 64, 81, 9, C.SPLIT_BF16, 0)
    try:
        for args in [(hb, 16, 64, 32, 64), (h, 16, 63, 32, 64), (h, 16, 64, 0, 64), (h, 0, 64, 32, 64),
                     (h, 4096, 64, 4096 + 8 * 64, 64)]:  # the last pair overlaps
            with pytest.raises(C.NeumannError) as e:
                C.neumann_eval_host(*args)
            assert e.value.code == C.EINVAL
    finally:
        C.neumann_plan_destroy(h)
        C.neumann_plan_destroy(hb)


def test_resident_orders_of_batched_plans():
    """Grouped batched plans hold their smallest orders in the resident launch:
    untuned, orders up to 48 (the most their shared memory holds is 52-60,
    by the scheme's matrices); none for FP64 or with NEUMANN_FLAG_NO_RESIDENT."""
    cases = [((81, 9, C.SPLIT_BF16, 0), 48), ((225, 15, C.SPLIT_FP16, 0), 48), ((81, 9, C.FP32, 0), 48),
             ((625, 25, C.SPLIT_BF16, 0), 48), ((81, 9, C.FP64, 0), 0), ((81, 9, C.SPLIT_BF16, C.FLAG_NO_RESIDENT), 0)]
    for (k, radix, dtype, flags), want in cases:
        h = C.neumann_plan_create_batched(100, 256, k, radix, dtype, flags)
        try:
            assert C.neumann_plan_info(h)["resident_max_n"] == want, (k, radix, dtype, flags)
        finally:
            C.neumann_plan_destroy(h)
    h = C.neumann_plan_create(64, 81, 9, C.SPLIT_BF16, 0)  # a single plan has none
    try:
        assert C.neumann_plan_info(h)["resident_max_n"] == 0
    finally:
        C.neumann_plan_destroy(h)
