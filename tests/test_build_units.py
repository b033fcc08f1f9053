"""The score kernel's launch shapes are compiled one per translation unit
(csrc/k_score_<threads>_<ctas>.cu), and a unit may choose the cooperative rasteriser's
candidate block width by defining B3D_CAND_X before it includes k_score.cuh. The shapes of
one thread count share template instantiations of the tile renderer, so they must agree on
the width (otherwise two definitions of one device function would differ between units),
and a definition placed after the include would have no effect. No GPU needed."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2312_08715_gb300", "csrc")
HEADER_DEFAULT = 2  # the width k_score.cuh uses when a unit defines none


def _cand_width(path):
    txt = open(path).read()
    inc = txt.index('#include "k_score.cuh"')
    m = re.search(r"^#define B3D_CAND_X (\d+)\s*$", txt, re.M)
    if m is None:
        return HEADER_DEFAULT
    assert m.start() < inc, f"{os.path.basename(path)} defines B3D_CAND_X after including k_score.cuh"
    return int(m.group(1))


def test_header_default_candidate_width():
    txt = open(os.path.join(CSRC, "k_score.cuh")).read()
    assert re.search(r"#ifndef B3D_CAND_X\s*\n#define B3D_CAND_X %d\b" % HEADER_DEFAULT, txt)


def test_shapes_of_one_thread_count_agree_on_the_candidate_width():
    units = sorted(glob.glob(os.path.join(CSRC, "k_score_*_*.cu")))
    by_nt = {}
    for u in units:
        m = re.match(r"k_score_(\d+)_(\d+)\.cu$", os.path.basename(u))
        assert m, u
        by_nt.setdefault(int(m.group(1)), set()).add(_cand_width(u))
    assert set(by_nt) == {32, 64, 128, 256}
    for nt, widths in by_nt.items():
        assert len(widths) == 1, f"{nt}-thread shapes disagree: {sorted(widths)}"
        (w,) = widths
        assert w in (1, 2, 4), (nt, w)


def test_other_users_of_the_tile_renderer_keep_the_default_width():
    # the gradient, noise-grid and materialised kernels include k_score.cuh with their own
    # visitors; a width defined there would change them without an A/B of their own
    for u in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        if re.match(r"k_score_\d+_\d+\.cu$", os.path.basename(u)):
            continue
        txt = open(u).read()
        if '#include "k_score.cuh"' in txt:
            assert "B3D_CAND_X" not in txt, os.path.basename(u)
