"""CPU check of the CTA-pair work schedule (xc_internal.h: pair_items,
pair_coords), the host/device function the pair kernel decodes its items
with.

Every lower block (r, c), r >= c, of a channel with nib block rows (Sec. 4.2's
lower-triangle blocks) must be computed exactly once: by a CTA whose row
block a and column block b are (r, c), or transposed, (a, b) = (c, r) with
a < b (the mirror block, stored conjugated).  At most one item of a channel
holds a single block.  A small C++ harness including the header runs the
function for nib = 1 .. 96 and prints every item; the test rebuilds the
coverage from that listing.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1107_4264_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "xc_internal.h"
int main() {
  for (int nib = 1; nib <= 96; ++nib) {
    const int n = xc::pair_items(nib);
    std::printf("nib %d %d\n", nib, n);
    for (int i = 0; i < n; ++i) {
      int a0, a1, b, single;
      xc::pair_coords(i, nib, &a0, &a1, &b, &single);
      std::printf("%d %d %d %d\n", a0, a1, b, single);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def listing(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("pair")
    src = d / "pair.cpp"
    src.write_text(HARNESS)
    exe = d / "pair"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    res, i = {}, 0
    while i < len(out) and out[i]:
        _, nib, n = out[i].split()
        nib, n = int(nib), int(n)
        items = [tuple(int(v) for v in out[i + 1 + k].split()) for k in range(n)]
        res[nib] = items
        i += 1 + n
    return res


def test_every_lower_block_exactly_once(listing):
    assert sorted(listing) == list(range(1, 97))
    for nib, items in listing.items():
        seen = {}
        singles = 0
        for a0, a1, b, single in items:
            assert 0 <= b < nib and 0 <= a0 < nib and 0 <= a1 < nib
            rows = [a0] if single else [a0, a1]
            singles += single
            if not single:
                assert a0 != a1
            for a in rows:
                blk = (a, b) if a >= b else (b, a)  # transposed: the mirror block
                seen[blk] = seen.get(blk, 0) + 1
        want = {(r, c) for r in range(nib) for c in range(r + 1)}
        assert set(seen) == want, nib
        assert all(v == 1 for v in seen.values()), nib
        assert singles <= 1
        # ceil(blocks / 2) items
        assert len(items) == (nib * (nib + 1) // 2 + 1) // 2


def test_large_n_schedule(listing):
    """N=256 x 2 pols (4 block rows, 10 blocks): five two-block items, no
    idle CTA; the leftovers (3, 1) and (3, 3) share column block 3."""
    items = listing[4]
    assert len(items) == 5 and not any(s for *_, s in items)
    assert (1, 3, 3, 0) in items or (3, 1, 3, 0) in items
