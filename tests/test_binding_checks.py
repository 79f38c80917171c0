"""Host-side argument checks of the Python binding (CPU, no GPU needed): a
sized buffer that is smaller than what a call would read or write raises
RF_ERR_ARG before the library is called, so a wrong allocation can never
reach a kernel."""
import numpy as np
import pytest

from paper_2605_30294_gb300 import rafi


def test_brick_sizes():
    # scalar bricks: (n/b)^3 bricks of (b+2)^3 x-y quads of 4 floats
    assert rafi.c0_bricks_floats(64, 32) == 8 * 34 ** 3 * 4
    assert rafi.c0_bricks_floats(1024, 128) == 512 * 130 ** 3 * 4
    # streamline bricks: (n/b)^3 bricks of (b+4)^3 x-pairs of 8 floats
    assert rafi.c2_bricks_floats(512, 128) == 64 * 132 ** 3 * 8


@pytest.mark.parametrize("short", ["volume", "bricks"])
def test_c0_make_bricks_refuses_short_buffers(short):
    n, b = 16, 8
    vol = np.zeros(n ** 3 - (1 if short == "volume" else 0), np.float32)
    bricks = np.zeros(rafi.c0_bricks_floats(n, b) - (1 if short == "bricks" else 0), np.float32)
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_c0_make_bricks(vol, n, b, bricks)
    assert e.value.status == rafi.RF_ERR_ARG and short in str(e.value)


def test_c2_make_bricks_refuses_the_scalar_brick_size():
    n, b = 16, 8
    field = np.zeros(n ** 3 * 3, np.float32)
    bricks = np.zeros(rafi.c0_bricks_floats(n, b), np.float32)  # a quarter of what the field needs
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_c2_make_bricks(field, n, b, bricks)
    assert e.value.status == rafi.RF_ERR_ARG


@pytest.mark.parametrize("call", ["rf_c0_march", "rf_c2_trace", "rf_c3_render", "rf_c4_render"])
def test_readers_refuse_short_bricks(call):
    n, b = 16, 8
    short = np.zeros(16, np.float32)
    with pytest.raises(rafi.RafiError) as e:
        if call == "rf_c0_march":
            rafi.rf_c0_march(0, short, n, b, short)
        elif call == "rf_c2_trace":
            rafi.rf_c2_trace(0, short, n, b, 0.25, 10, 0, short, 1)
        elif call == "rf_c3_render":
            rafi.rf_c3_render(0, short, [0.0] * 12, n, b, 4, 4, 1, 3, short, short)
        else:
            rafi.rf_c4_render(0, short, n, b, 1.0, [([0.0] * 12, 4, 4)], 1, 4, short)
    assert e.value.status == rafi.RF_ERR_ARG


@pytest.mark.parametrize("short", ["items", "items_out", "dest", "offsets_out", "stats_out"])
def test_static_partition_refuses_short_buffers(short):
    n, ib, R = 100, 48, 7
    bufs = dict(items=np.zeros(n * ib, np.uint8), items_out=np.zeros(n * ib, np.uint8),
                dest=np.zeros(n, np.int32), offsets_out=np.zeros(R + 1, np.int32), stats_out=np.zeros(4, np.int64))
    bufs[short] = bufs[short][:-1]
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_partition_static(bufs["items"], bufs["dest"], n, ib, R, bufs["items_out"], bufs["offsets_out"],
                                 bufs["stats_out"])
    assert e.value.status == rafi.RF_ERR_ARG and short in str(e.value)


@pytest.mark.parametrize("case", ["items_unaligned", "out_unaligned", "overlap", "in_place", "dest_unaligned",
                                  "offsets_unaligned", "stats_unaligned"])
def test_static_partition_refuses_misaligned_or_overlapping_pointers(case):
    # plain integers stand for device addresses: the library rejects them by
    # arithmetic alone and returns before any CUDA call, so no GPU is needed
    n, ib, R = 4, 16, 2
    items, out, dest, off, stats = 0x100000, 0x200000, 0x300000, 0x400000, 0x500000
    if case == "items_unaligned":
        items += 8
    elif case == "out_unaligned":
        out += 4
    elif case == "overlap":
        out = items + 16
    elif case == "in_place":
        out = items
    elif case == "dest_unaligned":
        dest += 2
    elif case == "offsets_unaligned":
        off += 1
    else:
        stats += 4
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_partition_static(items, dest, n, ib, R, out, off, stats)
    assert e.value.status == rafi.RF_ERR_ARG
    assert "aligned" in rafi.rf_last_error()


def test_wait_limits_refuse_a_null_context_and_wild_values():
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_set_wait_limits(0, 1000, 0)
    assert e.value.status == rafi.RF_ERR_ARG


def test_push_limit_refuses_a_null_context():
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_set_push_limit(0, 1 << 17)
    assert e.value.status == rafi.RF_ERR_ARG
    with pytest.raises(rafi.RafiError):
        rafi.rf_get_push_limit(0)


def test_rank_skew_refuses_a_null_context():
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_set_rank_skew(0, 4)
    assert e.value.status == rafi.RF_ERR_ARG
    with pytest.raises(rafi.RafiError):
        rafi.rf_get_rank_skew(0)


@pytest.mark.parametrize("short", ["items", "retired"])
def test_c1_joint_runs_refuse_short_buffers(short):
    # three runs of n items read 3 n items and retire into 3 n slots
    n = 100
    items = np.zeros((3 * n - (1 if short == "items" else 0), 16), np.uint32)
    retired = np.zeros((3 * n - (1 if short == "retired" else 0), 16), np.uint32)
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_c1_run_batched_runs(0, items, n, 1, [0, 1, 2], 1.1, (4, 4, 4), retired)
    assert e.value.status == rafi.RF_ERR_ARG and short in str(e.value)
