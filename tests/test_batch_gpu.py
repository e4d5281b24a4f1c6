"""GPU checks of the batched form: one persistent launch over several
subarrays, replayed from a CUDA graph, bit-exact against the int64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1107_4264_gb300 import build as engine_build
from paper_1107_4264_gb300 import synth, xc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    engine_build.build()
    xc.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def inputs(subs, npol, seed, lo=-127, hi=127):
    return [synth.uniform_int8((T, F, N, npol, 2), lo, hi, seed + 17 * i)
            for i, (N, F, T) in enumerate(subs)]


# Ragged station counts (partial 128-input blocks, a single-block subarray,
# N = 3), T not a multiple of 64, uneven channel counts.
SMALL = [(16, 4, 128), (40, 3, 200), (70, 2, 96), (3, 5, 64), (100, 2, 70)]


@pytest.mark.parametrize("npol", [2, 1])
def test_batch_bit_exact(npol, dev):
    xs = inputs(SMALL, npol, 500 + npol)
    bc = xc.BatchCorrelator(SMALL, npol=npol)
    try:
        outs = bc.correlate([x.to(dev) for x in xs], sync=True)
        for x, o in zip(xs, outs):
            np.testing.assert_array_equal(o.cpu().numpy(), oracle.correlate_i8(x.numpy()))
    finally:
        bc.close()


def test_batch_graph_replay_new_buffers_and_accumulate(dev):
    """Later calls replay the captured graph with new buffers; ACCUMULATE adds."""
    bc = xc.BatchCorrelator(SMALL, npol=2)
    try:
        a = inputs(SMALL, 2, 601)
        b = inputs(SMALL, 2, 602)
        outs_a = bc.correlate([x.to(dev) for x in a], sync=True)
        outs_b = bc.correlate([x.to(dev) for x in b], sync=True)
        for x, o in zip(b, outs_b):
            np.testing.assert_array_equal(o.cpu().numpy(), oracle.correlate_i8(x.numpy()))
        bc.set_option(xc.XC_OPT_ACCUMULATE, 1)
        bc.correlate([x.to(dev) for x in b], outs=outs_a, sync=True)
        for xa, xb, o in zip(a, b, outs_a):
            want = oracle.correlate_i8(xa.numpy()) + oracle.correlate_i8(xb.numpy())
            np.testing.assert_array_equal(o.cpu().numpy(), want)
    finally:
        bc.close()


def test_batch_tune_then_exact(dev):
    """The tuner times tile shape x packing x ring depth x order; the launch
    it keeps is bit-exact, and so is every forced candidate."""
    xs = [x.to(dev) for x in inputs(SMALL, 2, 700)]
    bc = xc.BatchCorrelator(SMALL, npol=2)
    try:
        outs = bc.new_outputs()
        ms, best = bc.tune(xs, outs, reps=2)
        assert 0 <= best < xc.XC_BATCH_CANDIDATES
        timed = [c for c, m in enumerate(ms) if m > 0]
        # every shape, both depths and all orders; packing only if a subarray packs
        assert {c // 12 for c in timed} == {0, 1, 2}
        assert {(c // 3) % 2 for c in timed} == {0, 1} and {c % 3 for c in timed} == {0, 1, 2}
        assert ms[best] == min(ms[c] for c in timed)
        outs = bc.correlate(xs, sync=True)
        want = [oracle.correlate_i8(x.cpu().numpy()) for x in xs]
        for w, o in zip(want, outs):
            np.testing.assert_array_equal(o.cpu().numpy(), w)
        # each tile shape forced in turn, through the captured graph
        for tile in (xc.XC_TILE_128, xc.XC_TILE_PAIR, xc.XC_TILE_WIDE):
            bc.set_option(xc.XC_OPT_TILE, tile)
            outs = bc.correlate(xs, sync=True)
            for w, o in zip(want, outs):
                np.testing.assert_array_equal(o.cpu().numpy(), w)
    finally:
        bc.close()


def test_batch_tuning_file(dev, tmp_path):
    """A tuning file records the winner; a second handle for the same batch
    applies it without timing anything, and stays exact."""
    path = str(tmp_path / "tune.txt")
    xs = [x.to(dev) for x in inputs(SMALL, 2, 300)]
    want = [oracle.correlate_i8(x.cpu().numpy()) for x in xs]
    bc = xc.BatchCorrelator(SMALL, npol=2)
    try:
        bc.set_cache(path)
        ms, best = bc.tune(xs, bc.new_outputs(), reps=1)
    finally:
        bc.close()
    key = xc.xc_batch_cache_key([s[0] for s in SMALL], [s[1] for s in SMALL], [s[2] for s in SMALL], 2,
                                xc.XC_CI8)
    assert xc.xc_batch_cache_lookup(path, key) == best
    bc = xc.BatchCorrelator(SMALL, npol=2)
    try:
        bc.set_cache(path)
        ms2, best2 = bc.tune(xs, bc.new_outputs(), reps=1)
        assert best2 == best
        assert [c for c, m in enumerate(ms2) if m >= 0] == [best]  # nothing else timed
        outs = bc.correlate(xs, sync=True)
        for w, o in zip(want, outs):
            np.testing.assert_array_equal(o.cpu().numpy(), w)
    finally:
        bc.close()


def test_batch_rejects_bad_use(dev):
    with pytest.raises(xc.XcError):
        xc.xc_batch_create([8, 0], [2, 2], [64, 64], 2, xc.XC_CI8)
    with pytest.raises(xc.XcError):
        xc.xc_batch_create([8] * 9, [2] * 9, [64] * 9, 2, xc.XC_CI8)
    with pytest.raises(xc.XcError):
        xc.xc_batch_create([8], [2], [64], 2, xc.XC_CF32)
    bc = xc.BatchCorrelator([(8, 2, 64)], npol=2)
    try:
        x = torch.zeros((64, 2, 8, 2, 2), dtype=torch.int8, device=dev)
        out = torch.zeros((2, 36, 4, 2), dtype=torch.int32, device=dev)
        assert xc.xc_correlate(bc.h, x.data_ptr(), out.data_ptr(), 0) == xc.XC_ERR_UNSUPPORTED
        assert xc.xc_batch_correlate(bc.h, [x.data_ptr() + 1], [out.data_ptr()], 0) == \
            xc.XC_ERR_ALIGNMENT
    finally:
        bc.close()


def _slice_check(x, out, N, c, lo, hi):
    """Channel c, stations [lo, hi): oracle of the station slice against the
    matching baselines of the full output."""
    xs = x[:, c:c + 1, lo:hi].cpu().numpy()
    want = oracle.correlate_i8(xs)[0]  # [nb_slice][P*P][2]
    s1, s2 = np.tril_indices(hi - lo)
    s1, s2 = s1 + lo, s2 + lo
    order = np.lexsort((s2, s1))  # slice baselines in k order
    k = s1[order] * (s1[order] + 1) // 2 + s2[order]
    got = out[c].cpu().numpy()[k]
    np.testing.assert_array_equal(got, want)


def test_batched_workload(dev):
    """The six-subarray workload (N = 32 ... 1024, 1.606e13 useful ops) in one
    launch: sampled whole channels against the oracle (two per subarray up to
    N = 384, one for N = 1024), every subarray against the single-subarray
    engine in full."""
    subs = [(w.nstation, w.nfreq, w.ntime) for w in synth.BATCHED]
    xs = [synth.int8_sky(w, device=dev) for w in synth.BATCHED]
    bc = xc.BatchCorrelator(subs, npol=2)
    try:
        outs = bc.correlate(xs, sync=True)
        rng = np.random.default_rng(31)
        for (N, F, T), x, o in zip(subs, xs, outs):
            if N <= 384:
                chans = sorted(rng.choice(F, size=2, replace=False).tolist())
                want = oracle.correlate_i8(x[:, chans].cpu().numpy())
                np.testing.assert_array_equal(o[chans].cpu().numpy(), want)
            else:
                # One whole channel of the N = 1024 subarray.  The oracle runs
                # in parallel over channels, so the channel's T samples are
                # cut into 16 time ranges presented as 16 channels; their
                # integer partial sums add up exactly.
                c = int(rng.integers(F))
                xc_ = x[:, c].cpu().numpy()  # [T][N][P][2]
                parts = xc_.reshape(16, T // 16, N, 2, 2).transpose(1, 0, 2, 3, 4)
                want = oracle.correlate_i8(np.ascontiguousarray(parts)).sum(axis=0)
                np.testing.assert_array_equal(o[c].cpu().numpy().astype(np.int64), want)
                _slice_check(x, o, N, c, 0, 48)
            eng = xc.Correlator(N, 2, F, T, "int8")
            try:
                single = eng.correlate(x, sync=True)
                assert torch.equal(single, o)
            finally:
                eng.close()
    finally:
        bc.close()
