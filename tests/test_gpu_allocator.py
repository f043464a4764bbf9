"""The device memory hook of vplbm_config (dev_alloc / dev_free), served by
PyTorch's caching allocator through vplbm.TorchAllocator.

The hook changes where the solver's buffers live, not what the kernels do, so
the bar is bitwise equality with a solver on the library's own pool, over
every buffer kind (populations, mask, solid velocity, outlet state, in-place
side arrays, momentum-exchange rings, staging buffers, checkpoint restore).
The accounting must balance: every block taken is given back, and PyTorch's
allocated bytes return to where they were. A failing or misaligned
allocation is refused with its status and leaves nothing behind.
"""
import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu

V = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global V
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import vplbm
    V = vplbm
    yield


NX, NY = 301, 70


def _bodies():
    return [I.BodySpec(150.5, 35.0, 9.0, amp_y=4.0, period=200.0, omega=0.002)]


def _config(storage, streaming, allocator=None, stream=None):
    return V.make_config(NX, NY, "mrt", storage, 0.62, bc="channel-convective", u_in=(0.04, 0.0),
                         ring_len=64, streaming=streaming, allocator=allocator, stream=stream)


def _run(cfg, n):
    """Every buffer kind: static mask with solid velocity, a moving rotating
    body, momentum-exchange records, host transfers both ways."""
    chi = I.random_mask(NX, NY, 71, 0.1)
    us = I.random_solid_velocity(NX, NY, 72, 0.03)
    s = V.Solver(cfg, _bodies())
    s.set_mask(chi, us)
    s.set_initial_velocity(I.velocity_field(NX, NY, (0.04, 0.0), 5e-3, seed=3))
    s.record_momentum_exchange(True)
    s.step(n)
    return s


def _results(s):
    return {"f": s.populations(), "forces": s.forces(), "mom": s.moments(),
            "me": s.momentum_exchange_forces(), "mask": s.mask()}


def _assert_same(a, b):
    assert np.array_equal(a["f"], b["f"])
    assert np.array_equal(a["mask"], b["mask"])
    for key in ("forces", "mom", "me"):
        for x, y in zip(a[key], b[key]):
            assert np.array_equal(x, y), key


@pytest.mark.parametrize("storage,streaming", [("f32", "ab"), ("f16", "aa"), ("f64", "aa")])
def test_torch_allocator_bitwise_and_balanced(storage, streaming):
    import torch
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    A = V.TorchAllocator()
    with _run(_config(storage, streaming), 7) as s:
        ref = _results(s)
        state = V.vplbm_save_state(s.h)
        s.step(5)
        ref_later = s.populations()
    cfg = _config(storage, streaming, allocator=A)
    with _run(cfg, 7) as s:
        assert A.allocs > 0 and A.frees < A.allocs
        assert A.live_bytes >= V.vplbm_footprint_bytes(cfg)
        assert torch.cuda.memory_allocated() - base >= A.live_bytes
        _assert_same(_results(s), ref)
    assert A.frees == A.allocs and A.live_bytes == 0
    # a restart from a checkpoint into a solver on the hook with the same
    # bodies (its solid-velocity field is allocated by the restore)
    with V.Solver(_config(storage, streaming, allocator=A), _bodies()) as d:
        V.vplbm_load_state(d.h, state)
        d.step(5)
        assert np.array_equal(d.populations(), ref_later)
    assert A.frees == A.allocs and A.live_bytes == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_grouped_solvers_on_the_hook():
    """Solvers whose buffers come from the hook step in one group (their
    shared stream is the allocator's) bitwise as they step alone."""
    import torch
    shared = torch.cuda.Stream()
    A = V.TorchAllocator(stream=shared)
    w1 = I.cylinder_channel(300, 75, 12.0, 0.05, 150.0, 0, xc=100.0, storage="f16", seed=7)
    w2 = I.cylinder_channel(200, 50, 8.0, 0.05, 100.0, 0, xc=60.0, storage="f32", seed=8)
    with V.Solver.from_workload(w1) as a, V.Solver.from_workload(w2) as b, \
            V.Solver.from_workload(w1, allocator=A) as c, \
            V.Solver.from_workload(w2, allocator=A, streaming="aa") as d:
        assert c.cfg.stream == d.cfg.stream == shared.cuda_stream
        a.step(23)
        b.step(11)
        V.vplbm_group_step([c.h, d.h], [23, 11])
        assert np.array_equal(a.populations(), c.populations())
        assert np.array_equal(b.populations(), d.populations())
    assert A.frees == A.allocs and A.live_bytes == 0


@pytest.mark.parametrize("storage,streaming,bc", [
    ("f32", "ab", "periodic"), ("f16", "aa", "channel-convective"), ("f64", "ab", "channel"),
    ("bf16", "aa", "channel"), ("f32", "aa", "periodic"), ("f16", "ab", "channel-convective")])
def test_footprint_is_what_creation_allocates(storage, streaming, bc):
    """vplbm_footprint_bytes (the serving admission figure) equals, to the
    byte, what vplbm_create takes through the hook."""
    A = V.TorchAllocator()
    cfg = V.make_config(1000, 333, "mrt", storage, 0.6, bc=bc, u_in=(0.05, 0.0), ring_len=777,
                        streaming=streaming, allocator=A)
    with V.Solver(cfg) as s:
        assert A.live_bytes == V.vplbm_footprint_bytes(cfg)
        s.step(2)
    assert A.live_bytes == 0


class _FailingAt(object):
    """Wraps a TorchAllocator so that its k-th allocation returns NULL."""

    def __init__(self, k):
        self.k = k
        self.inner = V.TorchAllocator()
        self.calls = 0
        inner_alloc = self.inner._do_alloc

        def alloc(nbytes, ctx):
            self.calls += 1
            return None if self.calls == self.k else inner_alloc(nbytes, ctx)

        self.inner._alloc = V.DEV_ALLOC_FN(alloc)

    def install(self, cfg):
        return self.inner.install(cfg)


def test_failing_allocation_is_nomem_and_leaves_nothing():
    """vplbm_create with the k-th allocation failing, for every k: NOMEM,
    every block already taken given back. An in-place solver with the
    convective outlet takes 12 buffers at creation (population store, mask,
    tile and group partials, counters, record ring, flag, solid box, outlet
    side copy, lost values, two outlet ghost states)."""
    created_with = None
    for k in range(1, 20):
        F = _FailingAt(k)
        cfg = _config("f32", "aa", allocator=F)
        try:
            s = V.Solver(cfg)
        except V.VplbmError as e:
            assert e.status == V.VPLBM_ERR_NOMEM
            assert F.inner.frees == F.inner.allocs == k - 1
            assert F.inner.live_bytes == 0
            continue
        with s:
            created_with = F.inner.allocs
            s.step(3)
        assert F.inner.frees == F.inner.allocs
        break
    assert created_with == 12


def test_misaligned_allocation_is_refused():
    """A dev_alloc that returns a pointer off the 256-byte grid: the block
    goes straight back through dev_free and vplbm_create fails with
    INVALID."""
    A = V.TorchAllocator()
    inner_alloc, inner_free = A._do_alloc, A._do_free

    def alloc(nbytes, ctx):
        p = inner_alloc(nbytes + 256, ctx)
        return None if p is None else p + 16

    def free(ptr, ctx):
        inner_free(ptr - 16, ctx)

    A._alloc = V.DEV_ALLOC_FN(alloc)
    A._free = V.DEV_FREE_FN(free)
    cfg = _config("f32", "ab", allocator=A)
    with pytest.raises(V.VplbmError) as e:
        V.Solver(cfg)
    assert e.value.status == V.VPLBM_ERR_INVALID
    assert A.allocs == A.frees == 1 and A.live_bytes == 0


def test_hook_refusals_need_no_device_work():
    """Only one of the two functions set: refused at creation; an allocator
    bound to another stream than the config's: refused by the binding."""
    import torch
    cfg = _config("f32", "ab")
    A = V.TorchAllocator()
    cfg.dev_alloc = A._alloc
    with pytest.raises(V.VplbmError) as e:
        V.vplbm_create(cfg)
    assert e.value.status == V.VPLBM_ERR_INVALID
    assert A.allocs == 0
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with pytest.raises(ValueError):
        _config("f32", "ab", allocator=V.TorchAllocator(stream=s1), stream=s2)
