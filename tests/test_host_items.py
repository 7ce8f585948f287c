"""Host-side work-item layout of a plan (no device): counting items.

The counting kernel's work is cut into units -- (field, chunk of the words of its block
bitmaps or of its wave bitmaps) -- and consecutive units of one candidate are packed into
counting items of at most 1024 pages (a page = 256 bitmap words) and at most 64 units.
These tests recompute that packing from the bitmap sizes the descriptor compiler reports
(`ws_describe_fields`) and compare it with the plan a batch would make (`ws_plan_dry_run`).
"""
import math

import pytest

from paper_2204_14242_gb300 import binding as B
from paper_2204_14242_gb300 import workloads as W
from test_oracle_pins import random_tiny

PAGE_WORDS = 256
PAGED_CHUNK = 262144      # words of a counting unit of a field whose pages the row walk flags
DENSE_CHUNK = 16384       # words of a counting unit otherwise (the default tuning)
ITEM_PAGES, ITEM_UNITS = 1024, 64


@pytest.fixture(scope="module", autouse=True)
def lib():
    try:
        B.load()
    except OSError as e:
        pytest.skip(f"library not built: {e}")


def units_of(config, hw, chunk):
    """Pages of every counting unit of one candidate, field by field, block part first."""
    out = []
    for f in B.ws_describe_fields(config, hw):
        for w in (int(f["words"][0]), int(f["words"][1])):
            for c0 in range(0, w, chunk):
                out.append(math.ceil(min(chunk, w - c0) / PAGE_WORDS))
    return out


def packed_items(pages):
    """Greedy packing of one candidate's units into counting items."""
    items, cur_pages, cur_units = 0, 0, 0
    for p in pages:
        if items == 0 or cur_pages + p > ITEM_PAGES or cur_units == ITEM_UNITS:
            items += 1
            cur_pages = cur_units = 0
        cur_pages += p
        cur_units += 1
    return items


def test_small_candidates_take_one_counting_item_each():
    """Units of one candidate share an item; no item holds two candidates' units."""
    hw = W.a100()
    rng = W.SplitMix64(808)
    cfgs = [random_tiny(rng) for _ in range(60)]
    info = B.ws_describe(cfgs, hw)
    want = 0
    for c, st in zip(cfgs, info["status"]):
        if st != B.WS_OK:
            continue
        pages = units_of(c, hw, PAGED_CHUNK)
        assert sum(pages) <= ITEM_PAGES and len(pages) <= ITEM_UNITS
        want += 1 if pages else 0
    assert want > 40
    assert B.ws_plan_dry_run(cfgs, hw, scratch_bytes=1 << 30)["count_items"] == want


def test_counting_items_hold_at_most_64_units():
    """A candidate of 40 small fields has 80 units: two items, although its pages are few."""
    N = (64, 16, 8)
    st = W.dense_strides(N)
    fields = [W.Field(8, [W.Access(0, 0, 0, 0)], strides=st) for _ in range(39)]
    fields.append(W.Field(8, [W.Access(0, 0, 0, 1)], strides=st))
    cfg = W.Config(N=N, B=(32, 2, 1), fields=fields)
    hw = W.a100()
    pages = units_of(cfg, hw, PAGED_CHUNK)
    assert len(pages) == 80 and sum(pages) <= ITEM_PAGES
    assert packed_items(pages) == 2
    assert B.ws_plan_dry_run([cfg], hw, scratch_bytes=1 << 30)["count_items"] == 2


@pytest.mark.parametrize("fold", [1, 2])
def test_counting_items_split_at_1024_pages(fold):
    """A large field's units pack greedily into items of at most 1024 pages; its bitmaps are
    far larger than one item.  Unfolded, the row walk fills them (units of 1024 pages);
    folded twice the wave bitmaps span 2^21 words or more, the group takes the segment walk
    and its units are 64-page chunks, sixteen to an item."""
    N = (1024, 1024, 256)
    f = W.Field(8, [W.Access(*o) for o in W.star_offsets(4)] + [W.Access(0, 0, 0, 1)], strides=W.dense_strides(N))
    cfg = W.Config(N=N, B=(4, 1, 64), fields=[f], fold_axis=2 if fold > 1 else 0, fold=fold)
    hw = W.a100()
    plan = B.ws_plan_dry_run([cfg], hw, scratch_bytes=8 << 30)
    assert (plan["row_items"] > 0) == (fold == 1)
    pages = units_of(cfg, hw, PAGED_CHUNK if fold == 1 else DENSE_CHUNK)
    assert sum(pages) > 4 * ITEM_PAGES
    assert plan["count_items"] == packed_items(pages)
    assert plan["count_items"] >= math.ceil(sum(pages) / ITEM_PAGES)


def test_batch_counting_items_add_up_per_candidate():
    """In a batch every candidate packs alone: the plan's items are the sum of each
    candidate's (25-point sweep shapes on a small domain, all row-walk fields)."""
    hw = W.a100()
    cfgs = W.stencil_25pt_sweep(N=(160, 128, 96))[::15]
    want = sum(packed_items(units_of(c, hw, PAGED_CHUNK)) for c in cfgs)
    assert B.ws_plan_dry_run(cfgs, hw, scratch_bytes=8 << 30)["count_items"] == want


def test_many_passes_keep_the_work_items():
    """Cutting a batch into many scratch passes moves no work item while every candidate's
    fields still fit one pass: passes break between candidates, and each candidate packs its
    own counting units alone (the layout packs each run of one candidate within one pass on
    its own, in parallel).  A pass smaller than a candidate splits its fields into several
    groups, each packed apart."""
    hw = W.a100()
    cfgs = W.stencil_25pt_sweep(N=(160, 128, 96))[::15]   # 4.7 MB of bitmaps, at most 305 KB a candidate
    want = sum(packed_items(units_of(c, hw, PAGED_CHUNK)) for c in cfgs)
    one = B.ws_plan_dry_run(cfgs, hw, scratch_bytes=8 << 30)
    many = B.ws_plan_dry_run(cfgs, hw, scratch_bytes=320 << 10)
    assert one["passes"] == 1 and many["passes"] >= 10
    for k in ("count_items", "enum_items", "row_items", "groups", "fields", "bitmap_bytes"):
        assert many[k] == one[k], k
    assert many["count_items"] == want
    split = B.ws_plan_dry_run(cfgs, hw, scratch_bytes=256 << 10)
    extra = split["groups"] - one["groups"]
    assert extra > 0 and split["count_items"] == want + extra
