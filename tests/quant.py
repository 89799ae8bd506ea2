"""Round-to-nearest-even emulation of the tensor-core operand types (BF16,
FP16, E4M3 with saturation), used by the tests to build the exact expected
result of a reduced-precision contraction from the oracle's FP64 normals."""
import numpy as np


def to_bf16(x):
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def to_fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def _e4m3_table():
    vals = []
    for e in range(16):
        for m in range(8):
            if e == 15 and m == 7:
                continue  # NaN encoding
            v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
            vals.append(v)
    t = np.array(sorted(set(vals)))
    return np.concatenate([-t[::-1], t[1:]]) if t[0] == 0 else np.concatenate([-t[::-1], t])


_E4M3 = _e4m3_table()
_E4M3_CODE = np.arange(_E4M3.size)


def to_e4m3(x):
    """Nearest E4M3 value, ties to the even mantissa, saturating at +-448."""
    x = np.clip(np.asarray(x, dtype=np.float64), -448.0, 448.0)
    idx = np.searchsorted(_E4M3, x)
    idx = np.clip(idx, 1, _E4M3.size - 1)
    lo, hi = _E4M3[idx - 1], _E4M3[idx]
    dlo, dhi = x - lo, hi - x
    pick_hi = dhi < dlo
    tie = dhi == dlo
    # even mantissa: the bit pattern's last mantissa bit; on this sorted grid
    # magnitudes alternate parity, so pick the candidate with even |code|.
    mag_code = lambda v: np.searchsorted(_E4M3[_E4M3 >= 0], np.abs(v))
    hi_even = (mag_code(hi) % 2) == 0
    pick_hi = np.where(tie, hi_even, pick_hi)
    return np.where(pick_hi, hi, lo)


def quantize(x, prec):
    return {"bf16": to_bf16, "fp16": to_fp16, "fp8": to_e4m3}[prec](x)
