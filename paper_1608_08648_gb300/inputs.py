"""Seeded synthetic inputs shared by the tests, the bench and the CPU oracle runs.

This module only draws input keys and payloads.  It holds none of the sorting
method's arithmetic (no sampling, no splitter choice, no classification), so the
CUDA path and the CPU oracle can both consume its arrays without sharing code.

Random numbers come from the counter-based form of SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
output of the stream keyed ``k`` is ``mix(k + (i + 1) * GAMMA)``, which is exactly
the (i+1)-th output of the sequential generator started from state ``k``.  A
stream is keyed by ``mix(seed + (stream_id + 1) * GAMMA)``.  Everything is
computed with wrapping int64 tensor arithmetic, so the same call gives the same
bits on the CPU and on a CUDA device.

The paper measures on random 32-byte strings (Section 3); its int32 / float64
analogue here is the ``uniform`` distribution.  The other named distributions
(Gaussian, all-zero, bucket-sorted, staggered, g-group, random duplicates) are
not defined in the paper; their recipes below are this project's definitions
and are documented with the design notes.
"""
from __future__ import annotations

import torch

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

# Stream identifiers (the sampling stream of the random splitter choice is 1;
# it is owned by the sorting code, not by this module).
S_UNIFORM = 11
S_GAUSS = 21            # 21..24: the four summed uniforms
S_BUCKET = 31
S_STAGGER = 41
S_GGROUP = 51
S_DUP_POOL = 61
S_DUP_PICK = 62
S_HOT_SEL = 71
S_HOT_POOL = 72
S_HOT_PICK = 73
S_KEY64 = 74
S_EDGE_KIND = 81
S_EDGE_BITS = 82
S_PAYLOAD = 91
S_SEGLEN = 101
S_ARRIVE = 111
S_REQKIND = 112
S_REQLEN = 113
S_REQOFF = 114
S_REQSEED = 115
S_STR = 121             # 121..124: the four words of a string
S_STR_POOL = 131
S_STR_PICK = 132

DISTRIBUTIONS = ("uniform", "gaussian", "zero", "bucket", "staggered", "ggroup", "dup")


def _s64(x: int) -> int:
    """Python int -> the int64 with the same low 64 bits."""
    x &= MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def mix64_int(z: int) -> int:
    """SplitMix64 output mix on a Python integer (reference form)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return mix64_int((seed + (stream + 1) * GAMMA) & MASK64)


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix_t(z: torch.Tensor) -> torch.Tensor:
    z = z ^ _lsr(z, 30)
    z = z * _s64(MIX1)
    z = z ^ _lsr(z, 27)
    z = z * _s64(MIX2)
    return z ^ _lsr(z, 31)


def u64(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Raw 64-bit outputs u(seed, stream, i) for int64 positions ``idx``.

    Returned as int64 tensors holding the unsigned bit pattern."""
    k = _s64(stream_key(seed, stream))
    z = (idx + 1) * _s64(GAMMA) + k
    return _mix_t(z)


def _positions(n: int, start: int, count: int | None, device) -> torch.Tensor:
    if count is None:
        count = n - start
    return torch.arange(start, start + count, dtype=torch.int64, device=device)


def _v31(seed, stream, i):
    """Uniform integers in [0, 2^31): the top 31 bits of u."""
    return _lsr(u64(seed, stream, i), 33)


def _unit(seed, stream, i):
    """Uniform doubles in [0, 1): the top 53 bits of u times 2^-53 (exact)."""
    return _lsr(u64(seed, stream, i), 11).to(torch.float64) * (2.0 ** -53)


def int_keys(dist: str, n: int, seed: int, p: int, start: int = 0, count: int | None = None,
             device="cpu") -> torch.Tensor:
    """int64 keys in [0, 2^31) for the named distribution, positions [start, start+count)."""
    i = _positions(n, start, count, device)
    if n == 0 or i.numel() == 0:
        return torch.zeros(0, dtype=torch.int64, device=device)
    W = (1 << 31) // p
    B = -(-n // p)                      # block length ceil(n/p)
    if dist == "uniform":
        return _v31(seed, S_UNIFORM, i)
    if dist == "gaussian":
        acc = torch.zeros_like(i)
        for t in range(4):
            acc = acc + _v31(seed, S_GAUSS + t, i)
        return acc >> 2
    if dist == "zero":
        return torch.zeros_like(i)
    if dist == "bucket":
        # p contiguous blocks; inside each, sub-block j (of p) is uniform in [jW, (j+1)W).
        o = i % B
        j = (o * p) // B
        return j * W + _v31(seed, S_BUCKET, i) % W
    if dist == "staggered":
        # block b is uniform in range index 2b+1 (b < p/2) or 2b-p (b >= p/2), width W.
        b = i // B
        half = p // 2
        r = torch.where(b < half, 2 * b + 1, 2 * b - p)
        r = r % p
        return r * W + _v31(seed, S_STAGGER, i) % W
    if dist == "ggroup":
        # g = 8: block b of group G = b // 8 has 8 sub-blocks; sub-block j is uniform in
        # range index (8G + p/2 + j) mod p, width W.
        g = 8
        b = i // B
        G = b // g
        o = i % B
        j = (o * g) // B
        r = (G * g + p // 2 + j) % p
        return r * W + _v31(seed, S_GGROUP, i) % W
    if dist == "dup":
        pool = _v31(seed, S_DUP_POOL, torch.arange(32, dtype=torch.int64, device=device))
        pick = _lsr(u64(seed, S_DUP_PICK, i), 1) % 32
        return pool[pick]
    raise ValueError(f"unknown distribution {dist!r}")


def narrow_i32_keys(n: int, lo: int, width: int, seed: int = 1, start: int = 0, count: int | None = None,
                    device="cpu") -> torch.Tensor:
    """int32 keys uniform in [lo, lo + width) (lo + width <= 2^31): inputs whose
    buckets span few distinct values."""
    i = _positions(n, start, count, device)
    return (lo + _v31(seed, S_UNIFORM, i) % width).to(torch.int32)


def keys(dist: str, n: int, dtype: str, seed: int = 1, p: int = 1024, start: int = 0,
         count: int | None = None, device="cpu") -> torch.Tensor:
    """Keys of type ``dtype`` in {'i32', 'u64', 'f64'} for a named distribution.

    i32: the integer recipe directly.  f64: uniform and Gaussian use 53-bit unit
    doubles; the structured distributions use int_key * 2^-31 (exact).
    u64: uniform 64-bit outputs for 'uniform', else the integer recipe widened."""
    if dtype == "i32":
        return int_keys(dist, n, seed, p, start, count, device).to(torch.int32)
    if dtype == "f64":
        i = _positions(n, start, count, device)
        if dist == "uniform":
            return _unit(seed, S_UNIFORM, i)
        if dist == "gaussian":
            acc = torch.zeros(i.shape, dtype=torch.float64, device=device)
            for t in range(4):
                acc = acc + _unit(seed, S_GAUSS + t, i)
            return acc * 0.25
        return int_keys(dist, n, seed, p, start, count, device).to(torch.float64) * (2.0 ** -31)
    if dtype == "u64":
        i = _positions(n, start, count, device)
        if dist == "uniform":
            return u64(seed, S_KEY64, i)
        return int_keys(dist, n, seed, p, start, count, device)
    raise ValueError(f"unknown dtype {dtype!r}")


def hot_u64_keys(n: int, seed: int = 2, start: int = 0, count: int | None = None,
                 device="cpu") -> torch.Tensor:
    """u64 keys (int64 bit patterns): uniform 64-bit values, except that position i is
    'hot' exactly when the top two bits of u(seed, HOT_SEL, i) are zero (probability
    1/4) and then copies pool[floor(h * 1000 / 2^32)], h the top 32 bits of
    u(seed, HOT_PICK, i), from a pool of 1000 values drawn from stream HOT_POOL."""
    i = _positions(n, start, count, device)
    if i.numel() == 0:
        return torch.zeros(0, dtype=torch.int64, device=device)
    pool = u64(seed, S_HOT_POOL, torch.arange(1000, dtype=torch.int64, device=device))
    hot = _lsr(u64(seed, S_HOT_SEL, i), 62) == 0
    pick = (_lsr(u64(seed, S_HOT_PICK, i), 32) * 1000) >> 32
    cold = u64(seed, S_KEY64, i)
    return torch.where(hot, pool[pick], cold)


def edge_f64_keys(n: int, seed: int = 7, start: int = 0, count: int | None = None,
                  device="cpu") -> torch.Tensor:
    """float64 keys mixing +0, -0, +inf, -inf, signed subnormals and signed normals.

    NaN is never produced (exponent 0x7FF only with a zero mantissa)."""
    i = _positions(n, start, count, device)
    if i.numel() == 0:
        return torch.zeros(0, dtype=torch.float64, device=device)
    kind = _lsr(u64(seed, S_EDGE_KIND, i), 61)          # 0..7
    bits = u64(seed, S_EDGE_BITS, i)
    sign = bits & _s64(1 << 63)
    mant = bits & ((1 << 52) - 1)
    exp = (_lsr(bits, 52) & 0x7FF) % 0x7FF              # 0..0x7FE: never inf/NaN
    normal = sign | (exp << 52) | mant
    sub = sign | torch.where(mant == 0, torch.ones_like(mant), mant)
    out = normal
    out = torch.where(kind == 0, torch.zeros_like(bits), out)                  # +0
    out = torch.where(kind == 1, torch.full_like(bits, _s64(1 << 63)), out)    # -0
    out = torch.where(kind == 2, torch.full_like(bits, 0x7FF << 52), out)      # +inf
    out = torch.where(kind == 3, torch.full_like(bits, _s64((0xFFF) << 52)), out)  # -inf
    out = torch.where(kind == 4, sub, out)                                     # subnormal
    return out.view(torch.float64)


def payload_index(n: int, start: int = 0, count: int | None = None, device="cpu") -> torch.Tensor:
    """The u32 payload 'original index' (held in an int32 tensor)."""
    return _positions(n, start, count, device).to(torch.int32)


def segment_lengths(nseg: int, lo: int = 1024, hi: int = 4194304, cap: int = 1 << 28,
                    seed: int = 3) -> tuple[torch.Tensor, float]:
    """Lengths of a batch of nseg arrays, log-uniform in [lo, hi): L_g = floor(lo *
    (hi/lo)^u_g), u_g the top 53 bits of u(seed, S_SEGLEN, g) as a unit double.

    When their total exceeds ``cap`` they are compressed in log space,
    L'_g = floor(lo * (L_g / lo)^gamma), with gamma the largest value in [0, 1]
    (60 bisection steps) whose total is <= cap; the spread of lengths shrinks
    but every length stays >= lo and the batch keeps nseg arrays.
    Returns (int64 lengths on the CPU, gamma)."""
    g = torch.arange(nseg, dtype=torch.int64)
    u = _unit(seed, S_SEGLEN, g)
    L = torch.floor(lo * torch.pow(torch.tensor(hi / lo, dtype=torch.float64), u))
    ratio = L / lo

    def lengths(gamma: float) -> torch.Tensor:
        return torch.floor(lo * torch.pow(ratio, gamma)).to(torch.int64)

    if int(L.sum().item()) <= cap:
        return L.to(torch.int64), 1.0
    a, b = 0.0, 1.0
    for _ in range(60):
        m = 0.5 * (a + b)
        if int(lengths(m).sum().item()) <= cap:
            a = m
        else:
            b = m
    return lengths(a), a


def segment_offsets(lengths: torch.Tensor) -> torch.Tensor:
    """Offsets [0, L_0, L_0 + L_1, ...] (int64, nseg + 1 entries)."""
    off = torch.zeros(lengths.numel() + 1, dtype=torch.int64)
    off[1:] = torch.cumsum(lengths.to(torch.int64), 0)
    return off


def serving_trace(count: int, rate: float = 2000.0, lo: int = 4096, hi: int = 1 << 26,
                  seed: int = 5) -> dict:
    """A trace of sort requests arriving as a Poisson process.

    Request i arrives at the sum of i + 1 exponential gaps -ln(1 - u)/rate (u the
    unit double of u(seed, S_ARRIVE, i)); the top two bits of u(seed, S_REQKIND, i)
    pick its key type (bit 63: float64, else int32) and values (bit 62: random
    duplicates, else uniform), each with probability 1/2; its length is
    log-uniform in [lo, hi) as in segment_lengths; its keys are the slice at
    offset floor(u * (hi - n + 1)) of a shared source array of hi keys of that
    type and distribution (so every input can stay resident on the device);
    its sample seed is u(seed, S_REQSEED, i).
    Returns CPU tensors / lists: arrival_s, dtype, dist, n, offset, req_seed."""
    g = torch.arange(count, dtype=torch.int64)
    gap = -torch.log1p(-_unit(seed, S_ARRIVE, g)) / rate
    arrival = torch.cumsum(gap, 0)
    kind = u64(seed, S_REQKIND, g)
    is_f64 = (kind < 0).tolist()                       # bit 63
    is_dup = (_lsr(kind, 62) & 1).bool().tolist()      # bit 62
    n = torch.floor(lo * torch.pow(torch.tensor(hi / lo, dtype=torch.float64),
                                   _unit(seed, S_REQLEN, g))).to(torch.int64)
    off = torch.floor(_unit(seed, S_REQOFF, g) * (hi - n + 1).to(torch.float64)).to(torch.int64)
    rseed = u64(seed, S_REQSEED, g)
    return {"arrival_s": arrival.tolist(), "dtype": ["f64" if f else "i32" for f in is_f64],
            "dist": ["dup" if d else "uniform" for d in is_dup], "n": n.tolist(), "offset": off.tolist(),
            "req_seed": [int(x) & MASK64 for x in rseed.tolist()], "lo": lo, "hi": hi}


STR_DISTRIBUTIONS = ("uniform", "dup", "prefix8", "prefix24", "ties16")


def strings(dist: str, n: int, seed: int = 1, start: int = 0, count: int | None = None,
            device="cpu") -> torch.Tensor:
    """32-byte string keys as a uint8 tensor of shape (count, 32).

    uniform : every byte uniform (the paper's workload, Section 3): word k of
              string i is u(seed, S_STR + k, i), stored little-endian.
    dup     : copies of 32 pool strings (pool word k of string j is
              u(seed, S_STR_POOL, 4 j + k)), string i picks pool[u(seed, S_STR_PICK, i) mod 32].
    prefix8 : the first 8 bytes equal for every string (pool word 0), the rest uniform.
    prefix24: the first 24 bytes equal (pool words 0-2), the last 8 uniform.
    ties16  : the first 16 bytes from one of 64 pool prefixes (picked as in dup),
              the last 16 uniform."""
    i = _positions(n, start, count, device)
    words = [u64(seed, S_STR + k, i) for k in range(4)]
    pool = u64(seed, S_STR_POOL, torch.arange(4 * 64, dtype=torch.int64, device=device)).view(64, 4)
    if dist == "uniform":
        pass
    elif dist == "dup":
        pick = _lsr(u64(seed, S_STR_PICK, i), 1) % 32
        words = [pool[pick, k] for k in range(4)]
    elif dist == "prefix8":
        words[0] = pool[0, 0].expand_as(i)
    elif dist == "prefix24":
        for k in range(3):
            words[k] = pool[0, k].expand_as(i)
    elif dist == "ties16":
        pick = _lsr(u64(seed, S_STR_PICK, i), 1) % 64
        words[0] = pool[pick, 0]
        words[1] = pool[pick, 1]
    else:
        raise ValueError(f"unknown string distribution {dist!r}")
    w = torch.stack([x.contiguous() for x in words], dim=1).contiguous()     # (count, 4) int64
    return w.view(torch.uint8).view(-1, 32)
