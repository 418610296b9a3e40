"""Argument checks of the Python binding.  CPU only: every case here is rejected before
a pointer crosses the ABI (the checks run in the order element type, rank, row width,
element count, then CUDA placement), so no context and no GPU are needed."""
import pytest
import torch


@pytest.fixture(scope="module")
def gbs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1104_2732_gb300 as g
    return g


@pytest.fixture
def ctx(gbs):
    c = object.__new__(gbs.Context)   # no gbs_create: the checks fire before any C call
    c._h = None
    c.device = 0
    return c


def test_require_checks_in_order(gbs):
    r = gbs._require
    f32 = torch.zeros(4, 36)
    with pytest.raises(TypeError, match="torch tensor"):
        r([1.0], "x")
    with pytest.raises(TypeError, match="float64"):
        r(f32, "F", dtype=torch.float64)
    with pytest.raises(ValueError, match="1-d"):
        r(f32, "F", dim=1)
    with pytest.raises(ValueError, match="rows of 35"):
        r(f32, "F", cols=35)
    with pytest.raises(ValueError, match="143 elements"):
        r(f32, "F", numel=143)
    with pytest.raises(ValueError, match="at least 145"):
        r(f32, "F", min_numel=145)
    with pytest.raises(TypeError, match="CUDA"):
        r(f32, "F", dtype=torch.float32, dim=2, cols=36, numel=144, min_numel=144)


def test_host_tensors_are_never_accepted(ctx):
    """No CPU fallback: a host tensor is refused by every entry point."""
    x = torch.zeros(100)
    for call in (lambda: ctx.select_kth(x, 1), lambda: ctx.median(x), lambda: ctx.array_stats(x),
                 lambda: ctx.cost_pass(x, 1, 0.0, 1.0), lambda: ctx.compact(x, 0.0, 1.0),
                 lambda: ctx.select_segmented(x, torch.tensor([0, 100])),
                 lambda: ctx.bracket_features(x), lambda: ctx.bracket_propose(x),
                 lambda: ctx.generate_training_array(x, 0),
                 lambda: ctx.knn_regress(x.view(25, 4), x, x.view(25, 4), 1),
                 lambda: ctx.knn_classify(x.view(25, 4), x.int(), 3, x.view(25, 4), 1)):
        with pytest.raises(TypeError, match="CUDA"):
            call()


def test_shapes_that_would_overrun_a_buffer_are_refused(ctx):
    # features must be rows of 36 (the kernels read 36 floats per row)
    with pytest.raises(ValueError, match="rows of 36"):
        ctx.bracket_forward(torch.zeros(8, 35))
    with pytest.raises(TypeError, match="float32"):
        ctx.bracket_forward(torch.zeros(8, 36, dtype=torch.float64))
    with pytest.raises(ValueError, match="2-d"):
        ctx.bracket_train(torch.zeros(36), torch.zeros(1), batch=1, steps=1)
    # counters come in whole 4-word blocks
    with pytest.raises(ValueError, match="multiple of 4"):
        ctx.philox(torch.zeros(10, dtype=torch.int32), torch.zeros(4, dtype=torch.int32))
    with pytest.raises(TypeError, match="int32"):
        ctx.philox(torch.zeros(8, dtype=torch.int64), torch.zeros(4, dtype=torch.int32))
    # regression operands
    with pytest.raises(TypeError, match="float32"):
        ctx.lms_lts(torch.zeros(10, 3, dtype=torch.float64), torch.zeros(10), torch.zeros(2, 3))
    with pytest.raises(ValueError, match="2-d"):
        ctx.lms_lts_fused(torch.zeros(30), torch.zeros(10), torch.zeros(2, 3))
    # kNN: float32 point and query rows
    with pytest.raises(TypeError, match="float32"):
        ctx.knn_regress(torch.zeros(10, 3, dtype=torch.float64), torch.zeros(10), torch.zeros(2, 3), 1)
    with pytest.raises(ValueError, match="2-d"):
        ctx.knn_classify(torch.zeros(30), torch.zeros(30, dtype=torch.int32), 2, torch.zeros(2, 3), 1)
    # segmented: float32 values, int64 offsets
    with pytest.raises(TypeError, match="float32"):
        ctx.select_segmented(torch.zeros(10, dtype=torch.float64), torch.tensor([0, 10]))


def test_unknown_configuration_keys_are_refused(ctx):
    with pytest.raises(TypeError, match="use_learnd"):
        ctx.set_config(use_learnd=1)
