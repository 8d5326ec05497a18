"""The exchange format of include/binning.h restated for the tests (no
binning arithmetic): IEEE totalOrder keys as int64, and a two-shard
workload whose attribute 2 is -0.0 on the first shard and +0.0 on the rest."""
import numpy as np


def encode_keys(v):
    """totalOrder keys as int64 (the exchange format): non-negative values
    keep their bits, negative ones flip the magnitude bits; f32 keys are
    sign-extended."""
    v = np.ascontiguousarray(v)
    if v.dtype == np.float64:
        b = v.view(np.int64)
        return np.where(b >= 0, b, b ^ np.int64(0x7FFFFFFFFFFFFFFF))
    b = v.view(np.int32)
    return np.where(b >= 0, b, b ^ np.int32(0x7FFFFFFF)).astype(np.int64)


def decode_keys(k, dtype):
    if dtype == np.float64:
        b = np.where(k >= 0, k, k ^ np.int64(0x7FFFFFFFFFFFFFFF))
        return b.astype(np.int64).view(np.float64)
    k32 = k.astype(np.int32)
    return np.where(k32 >= 0, k32, k32 ^ np.int32(0x7FFFFFFF)).astype(np.int32).view(np.float32)


def shard_workload(dtype, world=2):
    """Plummer particles; attribute 2 is -0.0 on the first rank's shard and
    +0.0 on the others, so every bin both shards reach has min -0.0 and max
    +0.0 only if the keys order -0 below +0."""
    import workloads
    w = workloads.plummer(90_001, seed=5, dtype=dtype, res=48)
    cut = np.linspace(0, w.n, world + 1).astype(int)[1]
    w.attrs[2] = np.where(np.arange(w.n) < cut, -0.0, 0.0).astype(dtype)
    return w


