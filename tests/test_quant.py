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
