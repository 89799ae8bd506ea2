"""The operand-rounding emulation used by the tensor-core parity tests agrees
with PyTorch's own float8_e4m3fn / bfloat16 / float16 conversions."""
import numpy as np
import pytest

from quant import to_bf16, to_e4m3, to_fp16


def test_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(100_000) * 50, np.linspace(-448, 448, 50_001),
                        rng.standard_normal(10_000) * 1e-3]).astype(np.float32)
    t = torch.from_numpy(x)
    assert np.array_equal(to_e4m3(x.astype(np.float64)), t.to(torch.float8_e4m3fn).double().numpy())
    assert np.array_equal(to_bf16(x), t.to(torch.bfloat16).double().numpy())
    assert np.array_equal(to_fp16(x), t.to(torch.float16).double().numpy())
    assert to_e4m3(np.array([1e6]))[0] == 448.0 and to_e4m3(np.array([-1e6]))[0] == -448.0


@pytest.mark.parametrize("prec,scheme", [("bf16", "log_euler"), ("fp16", "log_euler"), ("fp16", "euler"),
                                         ("fp8", "log_euler")])
def test_flip_bound_covers_planted_flips(orc, prec, scheme):
    """The reduced-precision parity tests allow each price to move by
    flip_bound for operands the kernel may round to the other code.  Plant
    the worst case in the emulation (every ambiguous operand at the other
    end of its window): every price moves by less than the bound, and the
    planted flips move some price by a visible fraction of it (the bound is
    not vacuous)."""
    from test_gpu_tc import _case, emulate, flip_bound, payoffs_from_U
    w, pays = _case(64, 3, 300, 8)
    U, aux = emulate(orc, w, prec, 300, 8, scheme, detail=True)
    Uf = emulate(orc, w, prec, 300, 8, scheme, flip=True)
    fb = flip_bound(aux, U, pays, w["r"], w["T"])
    base = payoffs_from_U(U, pays, w["r"], w["T"]).mean(axis=1)
    moved = payoffs_from_U(Uf, pays, w["r"], w["T"]).mean(axis=1)
    ratio = np.abs(moved - base) / np.array(fb)
    print(prec, scheme, "planted move / bound:", np.round(ratio, 3))
    assert np.all(ratio <= 1.0)
    assert ratio.max() >= 0.01
