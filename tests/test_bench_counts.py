"""The algorithmic counts behind the bench's roofline figures, pinned independently:
the U-Net's flops from the NumPy reference's layer table, the stencil's per-point
flops and bytes from the operation list of one fused iteration, and the k-pair
representatives of a Monkhorst-Pack mesh."""

import numpy as np

import bench
from oracle import unet as ref
from workloads.configs import monkhorst_pack


def test_unet_flops_match_the_reference_layer_table():
    nvox = 8 * 8 * 16
    levels = {"e1a": 0, "e1b": 0, "e2a": 1, "e2b": 1, "e3a": 2, "e3b": 2, "d2a": 1, "d2b": 1,
              "d1a": 0, "d1b": 0, "out": 0}
    want = sum(2 * 27 * cin * cout * nvox / 8 ** levels[name] for name, cin, cout, _ in ref.LAYERS)
    assert bench.unet_forward_flops(nvox, False) == want
    pad = lambda c: (c + 15) // 16 * 16  # noqa: E731
    want_pad = sum(2 * 27 * pad(cin) * pad(cout) * nvox / 8 ** levels[name] for name, cin, cout, _ in ref.LAYERS)
    assert bench.unet_forward_flops(nvox, True) == want_pad
    # the bench's own table is the reference's, level by level
    assert [(ci, co) for ci, co, _ in bench.UNET_LAYERS] == [(ci, co) for _, ci, co, _ in ref.LAYERS]


def test_stencil_counts():
    # order 2R: per neighbour pair and axis a complex add (2) and a complex
    # scale-accumulate (2 multiplies + 2 adds); diagonal (E - V + i Gamma) p: 6; the
    # on-the-fly p = r + beta p: 8; the pairing dot's complex multiply-add: 8
    for order in (2, 4, 6, 8, 10, 12):
        r = order // 2
        assert bench.stencil_flops_per_point(order) == 3 * r * 6 + 6 + 8 + 8
    assert bench.stencil_bytes_per_point(16) == 64 and bench.stencil_bytes_per_point(8) == 32


def test_k_pair_representatives_cover_the_mesh_once():
    kk, _ = monkhorst_pack(8, 8)
    reps = bench.k_representatives(kk)
    assert len(reps) == 32
    seen = set()
    for i in reps:
        a, b = kk[i]
        j = int(np.argmin(np.abs(kk[:, 0] + a) + np.abs(kk[:, 1] + b)))
        assert j not in reps  # the mirror -k is not itself a representative
        seen.update({i, j})
    assert seen == set(range(len(kk)))


def test_double_float_stencil_op_count():
    # FP32 operations of the double-float primitives: TwoSum 6, FastTwoSum 3, product
    # with FMA (1 multiply + 3 FMA) 4, lazy accumulation (TwoSum + 2 adds) 8, accurate
    # double-word sum (2 TwoSum + 2 FastTwoSum + 2 adds) 20
    two_sum, fast, prod, acc, dadd = 6, 3, 4, 8, 20
    cmul = 4 * prod + 2 * (two_sum + 2 + fast)  # complex double-float product
    p_update = cmul + 2 * dadd
    diagonal = dadd + 4 * prod + 4 * acc
    pair = two_sum + 2
    combine = 6 * acc + 2 * fast
    dot = 8 + 4 * prod + 4 * acc
    for order in (2, 4, 8, 12):
        r = order // 2
        want = p_update + diagonal + r * 6 * (pair + prod + acc) + combine + dot
        assert bench.stencil_df_ops_per_point(order) == want
        # equal spacings: per distance and component three pairs, two sums of them, one
        # product and one accumulation
        want_iso = p_update + diagonal + r * 2 * (3 * pair + 2 * pair + prod + acc) + combine + dot
        assert bench.stencil_df_ops_per_point(order, iso=True) == want_iso


def test_sketch_plan_is_seeded_and_in_range():
    kk, _ = monkhorst_pack(8, 8)
    reps = bench.k_representatives(kk)
    a = bench.sketch_plan(256, reps, 40, 16)
    b = bench.sketch_plan(256, reps, 40, 16)
    assert a == b
    assert bench.sketch_plan(256, reps, 7, 16) == a[:7]  # a step's window is independent of the count
    assert all(k in reps and 0 <= e <= 256 - 16 for k, e in a)
    assert len({k for k, _ in a}) > 5 and len({e for _, e in a}) > 10
