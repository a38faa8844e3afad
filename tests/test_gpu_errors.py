"""Status codes of the C ABI on a GPU: every error is reported, none traps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dense_inputs(m=200, d=10, n=300, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (torch.from_numpy(rng.standard_normal((m, d)).astype(np.float32)).cuda(),
            torch.from_numpy(rng.standard_normal((d, n)).astype(np.float32)).cuda())


def test_sample_before_tables_is_a_state_error():
    import paper_1506_03872_gb300 as mad
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_sample(c.ctx, 10, 1)
        assert e.value.status == mad.MAD_ERR_STATE


def test_bad_flags_and_shapes():
    import paper_1506_03872_gb300 as mad
    with pytest.raises(mad.MadError) as e:
        mad.mad_create(64)
    assert e.value.status == mad.MAD_ERR_ARG
    A, B = _dense_inputs()
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(B[:5]), 100)
        assert e.value.status == mad.MAD_ERR_ARG
        with pytest.raises(mad.MadError) as e:
            mad.mad_set_hash_capacity(c.ctx, 1000)   # not a power of two
        assert e.value.status == mad.MAD_ERR_ARG


def test_zero_matrix_is_empty():
    import paper_1506_03872_gb300 as mad
    A, B = _dense_inputs()
    A.zero_()
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(B), 100)
        assert e.value.status == mad.MAD_ERR_EMPTY


def test_more_diamonds_than_s_max_overflows():
    import paper_1506_03872_gb300 as mad
    A, B = _dense_inputs()
    with mad.Context() as c:
        mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(B), 1000)
        mad.mad_sample(c.ctx, 600, 1)
        with pytest.raises(mad.MadError) as e:
            mad.mad_sample(c.ctx, 600, 1, 600)
        assert e.value.status == mad.MAD_ERR_OVERFLOW
        mad.mad_reset_hash(c.ctx)
        mad.mad_sample(c.ctx, 1000, 1)      # allowed again after a reset


def test_hash_too_small_reports_hash_full():
    import paper_1506_03872_gb300 as mad
    A, B = _dense_inputs(m=2000, n=3000)
    with mad.Context() as c:
        mad.mad_set_hash_capacity(c.ctx, 1024)
        mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(B), 100_000)
        mad.mad_sample(c.ctx, 100_000, 1)
        with pytest.raises(mad.MadError) as e:
            mad.mad_topk(c.ctx, 10)
        assert e.value.status == mad.MAD_ERR_HASH_FULL
        assert mad.mad_stats(c.ctx)["device_error"] != 0
    # the device stays usable
    x = torch.ones(4, device="cuda")
    assert float(x.sum()) == 4.0


def test_unsupported_mixed_formats():
    import paper_1506_03872_gb300 as mad
    A, B = _dense_inputs()
    rowptr = torch.zeros(11, dtype=torch.int64, device="cuda")
    colidx = torch.zeros(1, dtype=torch.int32, device="cuda")
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_build_tables(c.ctx, mad.dense(A), mad.csr(rowptr, colidx, (10, 300)), 100)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED


def test_phase_events_bracket_the_sampling_kernels():
    import paper_1506_03872_gb300 as mad
    A, B = _dense_inputs(m=2000, d=20, n=3000)
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_set_phase_events(c.ctx, [torch.cuda.Event(enable_timing=True) for _ in range(5)])
        assert e.value.status == mad.MAD_ERR_ARG
        mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(B), 200000)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        outer = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        mad.mad_set_phase_events(c.ctx, ev)
        outer[0].record()
        mad.mad_sample(c.ctx, 200000, 7)
        outer[1].record()
        mad.mad_set_phase_events(c.ctx, [])
        torch.cuda.synchronize()
        parts = [ev[q].elapsed_time(ev[q + 1]) for q in range(3)]
        assert all(p >= 0.0 for p in parts)
        assert sum(parts) <= outer[0].elapsed_time(outer[1]) + 1e-3
        assert mad.mad_stats(c.ctx)["inserted"] > 0


def test_square_sym_needs_01_gram_inputs():
    import paper_1506_03872_gb300 as mad
    A, B = _dense_inputs()
    with mad.Context(2 | 8) as c:   # dense inputs: not built for Sec. 3.2.3
        with pytest.raises(mad.MadError) as e:
            mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(A.T.contiguous()), 100)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED


@pytest.mark.parametrize("nth", [1, 2, 5])
def test_injected_allocation_failure_returns_oom(monkeypatch, nth):
    """Host-side fault injection (no GPU fault): with MAD_FAULT=oom:N at
    context creation, the context's N-th device allocation and every later
    one fail, and the call that needs them returns MAD_ERR_OOM; the context
    is destroyed cleanly and a context created without the variable works
    on the same device."""
    import paper_1506_03872_gb300 as mad
    rng = np.random.Generator(np.random.PCG64(90))
    A = torch.from_numpy(rng.standard_normal((300, 20)).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal((20, 400)).astype(np.float32)).cuda()
    monkeypatch.setenv("MAD_FAULT", f"oom:{nth}")
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(B), 50_000)
        assert e.value.status == mad.MAD_ERR_OOM
        with pytest.raises(mad.MadError) as e:
            mad.mad_dense_topt(c.ctx, mad.dense(A), mad.dense(B), 10)
        assert e.value.status == mad.MAD_ERR_OOM
    monkeypatch.delenv("MAD_FAULT")
    with mad.Context() as c:
        mad.mad_build_tables(c.ctx, mad.dense(A), mad.dense(B), 50_000)
        mad.mad_sample(c.ctx, 50_000, 3)
        _, n = mad.mad_topk(c.ctx, 100)
        assert n == 100
