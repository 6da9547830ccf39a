"""Device-mode argument checks of the Python binding, on CPU.

The C ABI receives plain device pointers and cannot see a buffer's size or
type, so the binding checks each device tensor (CUDA, on the context's device,
dtype, element count, contiguity) before the call.  These tests drive those
checks with a stand-in tensor object and a recording stand-in library: a
rejected argument never reaches the library, an accepted one passes its
data pointer through unchanged."""
import types

import numpy as np
import pytest

from paper_1701_03549_gb300 import fire


class FakeTensor:
    """The attributes of a torch tensor that the binding's checks read."""

    def __init__(self, dtype, shape, device=0, cuda=True, contiguous=True,
                 ptr=0x10000):
        self.dtype = f"torch.{dtype}"
        self.shape = tuple(shape)
        self.device = types.SimpleNamespace(index=device)
        self.is_cuda = cuda
        self._contig = contiguous
        self._ptr = ptr

    def numel(self):
        return int(np.prod(self.shape, dtype=np.int64))

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        return self._ptr


class FakeLib:
    """Records the calls that reach the library; every call succeeds."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append((name, args))
            return fire.FIRE_OK
        return f


class FakeCtx:
    def __init__(self, device=0):
        self.lib = FakeLib()
        self.h = 1
        self.device = device

    def check(self, rc):
        return rc


@pytest.fixture(autouse=True)
def fake_tensors(monkeypatch):
    real = fire._is_tensor
    monkeypatch.setattr(fire, "_is_tensor",
                        lambda a: isinstance(a, FakeTensor) or real(a))


def _fitness_args(n=4, **over):
    a = dict(results=FakeTensor("int32", (n, 6), ptr=0x1000),
             out=FakeTensor("float64", (n,), ptr=0x2000))
    a.update(over)
    return a


def test_valid_device_arguments_reach_the_library():
    ctx = FakeCtx()
    a = _fitness_args()
    fire.fire_fitness(ctx, a["results"], 1, device=True, out=a["out"])
    (name, args), = ctx.lib.calls
    assert name == "fire_fitness"
    assert args == (1, 0x1000, 4, 1, fire.FIRE_DEVICE_PTRS, 0x2000)


@pytest.mark.parametrize("bad,what", [
    (FakeTensor("float64", (3,)), "elements"),                 # short
    (FakeTensor("float64", (5,)), "elements"),                 # long
    (FakeTensor("float32", (4,)), "dtype"),
    (FakeTensor("float64", (4,), cuda=False), "CUDA"),
    (FakeTensor("float64", (4,), device=1), "cuda:1"),
    (FakeTensor("float64", (4,), contiguous=False), "contiguous"),
    (None, "required"),
])
def test_bad_output_is_rejected_before_the_call(bad, what):
    ctx = FakeCtx()
    a = _fitness_args(out=bad)
    with pytest.raises(fire.FireError) as e:
        fire.fire_fitness(ctx, a["results"], 0, device=True, out=a["out"])
    assert e.value.code == fire.FIRE_EINVAL and what in str(e.value)
    assert ctx.lib.calls == []


def test_results_need_six_words_per_row():
    ctx = FakeCtx()
    with pytest.raises(fire.FireError):
        fire.fire_fitness(ctx, FakeTensor("int32", (4, 5)), 0, device=True,
                          out=FakeTensor("float64", (4,)))
    # the uint32 bit pattern is accepted as well
    fire.fire_fitness(ctx, FakeTensor("uint32", (4, 6)), 0, device=True,
                      out=FakeTensor("float64", (4,)))
    assert len(ctx.lib.calls) == 1


def _map(ctx, H=20, W=30):
    m = fire.Map.__new__(fire.Map)
    m.ctx, m.h, m.H, m.W = ctx, 7, H, W
    return m


def _batch(n, H=20, W=30, **over):
    a = dict(params=FakeTensor("float64", (n, 5)),
             ignitions=FakeTensor("int32", (n, 2)),
             seeds=FakeTensor("int64", (n,)),
             out=FakeTensor("int32", (n, 6)),
             burn_step=None)
    a.update(over)
    return a


def test_simulate_batch_checks_every_buffer():
    ctx = FakeCtx()
    m = _map(ctx)
    m.simulate_batch(**_batch(8), device=True)
    m.simulate_batch(**_batch(8, burn_step=FakeTensor("int32", (8, 20, 30))),
                     device=True, want_steps=True)
    assert len(ctx.lib.calls) == 2
    for over in (dict(params=FakeTensor("float32", (8, 5))),
                 dict(params=FakeTensor("float64", (8, 4))),
                 dict(ignitions=FakeTensor("int64", (8, 2))),
                 dict(seeds=FakeTensor("int32", (8,))),
                 dict(seeds=FakeTensor("int64", (7,))),
                 dict(out=FakeTensor("int32", (8, 5))),
                 dict(burn_step=FakeTensor("int32", (8, 20, 29)))):
        with pytest.raises(fire.FireError):
            m.simulate_batch(**_batch(8, **over), device=True)
    with pytest.raises(fire.FireError):      # steps wanted, no buffer
        m.simulate_batch(**_batch(8), device=True, want_steps=True)
    assert len(ctx.lib.calls) == 2


def test_burnout_checks_the_burn_time_plane():
    ctx = FakeCtx()
    m = _map(ctx)
    m.simulate_burnout(burn_time=FakeTensor("uint8", (20, 30)), device=True,
                       **{k: v for k, v in _batch(3).items()})
    with pytest.raises(fire.FireError):
        m.simulate_burnout(burn_time=FakeTensor("uint8", (30, 20, 2)),
                           device=True, **_batch(3))
    assert len(ctx.lib.calls) == 1


def test_ga_step_and_group_mean_sizes():
    ctx = FakeCtx()
    P, G = 6, 5
    g = dict(genes=FakeTensor("float64", (P, G), ptr=0x100),
             fitness=FakeTensor("float64", (P,)),
             lo=FakeTensor("float64", (G,)), hi=FakeTensor("float64", (G,)))
    fire.ga_step(ctx, g["genes"], g["fitness"], 0, 10, 1, g["lo"], g["hi"],
                 device=True, out=FakeTensor("float64", (P, G), ptr=0x900))
    with pytest.raises(fire.FireError):
        fire.ga_step(ctx, g["genes"], g["fitness"], 0, 10, 1, g["lo"],
                     FakeTensor("float64", (G - 1,)), device=True,
                     out=FakeTensor("float64", (P, G)))
    fire.fire_group_mean(ctx, FakeTensor("float64", (24,)), 4, device=True,
                         out=FakeTensor("float64", (6,)))
    with pytest.raises(fire.FireError):      # 25 values: not whole groups
        fire.fire_group_mean(ctx, FakeTensor("float64", (25,)), 4,
                             device=True, out=FakeTensor("float64", (6,)))
    assert [c[0] for c in ctx.lib.calls] == ["ga_step", "fire_group_mean"]


def test_multi_and_tc_gemm_sizes():
    ctx = FakeCtx()
    n = 5
    a = _batch(n)
    fire.fire_simulate_multi(ctx, [], FakeTensor("int32", (n,)), a["params"],
                             a["ignitions"], a["seeds"], device=True,
                             out=a["out"])
    with pytest.raises(fire.FireError):
        fire.fire_simulate_multi(ctx, [], FakeTensor("int64", (n,)),
                                 a["params"], a["ignitions"], a["seeds"],
                                 device=True, out=a["out"])
    fire.fire_tc_gemm(ctx, FakeTensor("bfloat16", (128, 64)),
                      FakeTensor("bfloat16", (96, 64)), 128, 96, 64,
                      FakeTensor("float32", (128, 96)))
    with pytest.raises(fire.FireError):      # float16 is not bfloat16
        fire.fire_tc_gemm(ctx, FakeTensor("float16", (128, 64)),
                          FakeTensor("bfloat16", (96, 64)), 128, 96, 64,
                          FakeTensor("float32", (128, 96)))
    assert [c[0] for c in ctx.lib.calls] == ["fire_simulate_multi",
                                             "fire_tc_gemm"]


def test_host_rasters_must_share_one_shape():
    ctx = FakeCtx()
    ctx.lib = FakeLib()
    veg = np.ones((4, 5), np.uint8)
    f = np.zeros((4, 5), np.float32)
    with pytest.raises(fire.FireError):
        fire.Context.maps_upload(ctx, veg, f, f, np.zeros((5, 4), np.float32),
                                 f)
    assert ctx.lib.calls == []
