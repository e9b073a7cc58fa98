"""Seeded synthetic inputs for the closed-shell (T) correction.

This module only draws random numbers and assembles integral blocks from a
density-fitting factor; it holds none of the (T) arithmetic (no W, V, D or
energy).  Both the CPU oracle and the GPU library are fed from here.

Recipe (the paper prints no inputs; these follow the workload description of
its synthetic stand-ins):

* orbital energies: occupied ~ U[-1.5, -0.3] Eh, virtual ~ U[0.1, 3.0] Eh,
  each sorted ascending, occupied first;
* density-fitting factor B[Q, p, q] ~ N(0, 0.05), symmetric in (p, q), with
  Q = 3 (o + v); every value is rounded to a multiple of 2**-20 (|B| clipped
  to 0.5) so that each integral (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s] is an exact
  binary number: any summation order (CPU or GPU) gives the same bits;
* t1[i, a] ~ N(0, 0.005);
* t2[i, j, a, b] ~ N(0, 0.01) with t2[i, j, a, b] = t2[j, i, b, a].

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based
generator -- draw n of a stream is the SplitMix64 finaliser applied to
seed + (n + 1) * 0x9E3779B97F4A7C15 -- mapped to 53-bit uniforms, and
Box-Muller (1958) normals (cosine branch, two uniforms per normal).  Each
array has its own stream (the run seed mixed with a per-array tag), so the
value of an element depends only on (seed, array, element index).
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

TAG_EPS_OCC, TAG_EPS_VIR, TAG_B, TAG_T1, TAG_T2 = 1, 2, 3, 4, 5

B_SIGMA, T1_SIGMA, T2_SIGMA = 0.05, 0.005, 0.01
B_GRID = 2.0 ** -20
B_CLIP = 0.5

# Seeds of the five named workloads: index k -> 20251201 + k.
CONFIG_SEED_BASE = 20251201

WORKLOADS = {
    # name: (o, v)
    "tiny_o6_v36": (6, 36),
    "single_o20_v200": (20, 200),
    "precision_o40_v400": (40, 400),
    "large_o50_v450": (50, 450),
}
WORKLOAD_SEEDS = {
    "tiny_o6_v36": CONFIG_SEED_BASE + 0,
    "single_o20_v200": CONFIG_SEED_BASE + 1,
    "precision_o40_v400": CONFIG_SEED_BASE + 2,
    "large_o50_v450": CONFIG_SEED_BASE + 4,
}
SERVING_SEED_BASE = 31000000
SERVING_ARRIVAL_SEED = 4242


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, tag: int) -> np.uint64:
    """Seed of the per-array stream: the finaliser of (seed, tag)."""
    s = np.array([(int(seed) * 0x100000001B3 + int(tag) * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _mix(s)[0]


def raw_u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream (seed, tag)."""
    s0 = stream_seed(seed, tag)
    n = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(s0 + n * _GOLDEN)


def uniform(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    return (raw_u64(seed, tag, start, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Standard normals; normal n uses uniforms 2n and 2n+1 (Box-Muller, cosine branch)."""
    u = uniform(seed, tag, 2 * start, 2 * count)
    u1 = 1.0 - u[0::2]          # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass
class Amplitudes:
    """Orbital energies, DF factor and CCSD-like amplitudes of one synthetic job."""
    o: int
    v: int
    seed: int
    eps: np.ndarray      # [o + v], occupied first
    B: np.ndarray        # [Q, o + v, o + v], symmetric in the last two indices
    t1: np.ndarray       # [o, v]
    t2: np.ndarray       # [o, o, v, v]

    @property
    def Q(self) -> int:
        return self.B.shape[0]


def _draw_symmetric_B(seed: int, Q: int, N: int) -> np.ndarray:
    iu, ju = np.triu_indices(N)
    npair = iu.size
    B = np.empty((Q, N, N), dtype=np.float64)
    for q in range(Q):
        x = normal(seed, TAG_B, q * npair, npair) * B_SIGMA
        x = np.clip(np.rint(x / B_GRID) * B_GRID, -B_CLIP, B_CLIP)
        B[q, iu, ju] = x
        B[q, ju, iu] = x
    return B


def _draw_t2(seed: int, o: int, v: int) -> np.ndarray:
    ov = o * v
    t2m = np.empty((ov, ov), dtype=np.float64)
    chunk_rows = max(1, (1 << 24) // max(ov, 1))
    # Upper triangle (I <= J) of the (i a) x (j b) matrix, row by row, drawn in
    # row-major order of the triangle; the lower triangle is the mirror.
    base = 0
    for r0 in range(0, ov, chunk_rows):
        r1 = min(ov, r0 + chunk_rows)
        lens = ov - np.arange(r0, r1)
        total = int(lens.sum())
        x = normal(seed, TAG_T2, base, total) * T2_SIGMA
        off = 0
        for r, ln in zip(range(r0, r1), lens):
            t2m[r, r:] = x[off:off + ln]
            t2m[r:, r] = x[off:off + ln]
            off += ln
        base += total
    # t2m[(i a), (j b)] -> t2[i, j, a, b]
    return t2m.reshape(o, v, o, v).transpose(0, 2, 1, 3).copy()


def make_amplitudes(o: int, v: int, seed: int, Q: int | None = None) -> Amplitudes:
    """Draw one job: eps, B, t1, t2 (the integral blocks are built from B on demand)."""
    if o < 1 or v < 1:
        raise ValueError("o and v must be positive")
    N = o + v
    if Q is None:
        Q = 3 * N
    eps_o = np.sort(-1.5 + 1.2 * uniform(seed, TAG_EPS_OCC, 0, o))
    eps_v = np.sort(0.1 + 2.9 * uniform(seed, TAG_EPS_VIR, 0, v))
    eps = np.concatenate([eps_o, eps_v])
    B = _draw_symmetric_B(seed, Q, N)
    t1 = (normal(seed, TAG_T1, 0, o * v) * T1_SIGMA).reshape(o, v)
    t2 = _draw_t2(seed, o, v)
    return Amplitudes(o=o, v=v, seed=seed, eps=eps, B=B, t1=t1, t2=t2)


# ---------------------------------------------------------------------------
# Integral blocks (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s]   (Mulliken notation)
# Layouts used throughout the library:
#   ovvv[i, a, b, d] = (ia|bd)      [o, v, v, v]
#   ovoo[i, a, j, l] = (ia|jl)      [o, v, o, o]
#   ovov[i, a, j, b] = (ia|jb)      [o, v, o, v]
# ---------------------------------------------------------------------------

def _B_blocks(amp: Amplitudes):
    o = amp.o
    Bov = amp.B[:, :o, o:]
    Bvv = amp.B[:, o:, o:]
    Boo = amp.B[:, :o, :o]
    return Bov, Bvv, Boo


def ovvv_slice(amp: Amplitudes, i: int) -> np.ndarray:
    """(ia|bd) for one occupied i: [v, v, v]."""
    Bov, Bvv, _ = _B_blocks(amp)
    Q, v = amp.Q, amp.v
    return (Bov[:, i, :].T @ Bvv.reshape(Q, v * v)).reshape(v, v, v)


def ovvv(amp: Amplitudes) -> np.ndarray:
    Bov, Bvv, _ = _B_blocks(amp)
    Q, o, v = amp.Q, amp.o, amp.v
    return (Bov.reshape(Q, o * v).T @ Bvv.reshape(Q, v * v)).reshape(o, v, v, v)


def ovoo(amp: Amplitudes) -> np.ndarray:
    Bov, _, Boo = _B_blocks(amp)
    Q, o, v = amp.Q, amp.o, amp.v
    return (Bov.reshape(Q, o * v).T @ Boo.reshape(Q, o * o)).reshape(o, v, o, o)


def ovov(amp: Amplitudes) -> np.ndarray:
    Bov, _, _ = _B_blocks(amp)
    Q, o, v = amp.Q, amp.o, amp.v
    X = Bov.reshape(Q, o * v)
    return (X.T @ X).reshape(o, v, o, v)


@dataclasses.dataclass
class Job:
    """Everything the (T) energy needs, as host arrays (C-contiguous float64)."""
    o: int
    v: int
    eps: np.ndarray
    t1: np.ndarray
    t2: np.ndarray
    ovvv: np.ndarray
    ovoo: np.ndarray
    ovov: np.ndarray


def make_job(o: int, v: int, seed: int, Q: int | None = None) -> Job:
    """A complete small job on the host (ovvv is o*v^3 doubles: keep v modest)."""
    amp = make_amplitudes(o, v, seed, Q)
    return Job(o=o, v=v, eps=amp.eps, t1=amp.t1, t2=amp.t2,
               ovvv=ovvv(amp), ovoo=ovoo(amp), ovov=ovov(amp))


def workload_job(name: str) -> Job:
    o, v = WORKLOADS[name]
    return make_job(o, v, WORKLOAD_SEEDS[name])


def serving_request_shape(r: int) -> tuple[int, int]:
    """(o, v) of serving request r: o ~ U{6..32}, v = round(o * U[6, 12])."""
    u = uniform(SERVING_SEED_BASE + r, 99, 0, 2)
    o = 6 + int(u[0] * 27)
    v = int(round(o * (6.0 + 6.0 * u[1])))
    return o, v


# ---------------------------------------------------------------------------
# The same generator on a CUDA device (serving streams of hundreds of jobs,
# where drawing hundreds of millions of numbers on the host would dominate).
# SplitMix64 runs in 64-bit integer arithmetic (wrapping multiplications,
# logical shifts built from arithmetic ones), so the raw draws and the
# uniforms are bit-identical to the host generator's; the Box-Muller normals
# use the device's log and cos and may differ from the host's in the last
# place, and so may (rarely) a factor value rounded to the 2^-20 grid.
# ---------------------------------------------------------------------------

def _to_i64(x: int) -> int:
    x &= 0xFFFFFFFFFFFFFFFF
    return x - (1 << 64) if x >= (1 << 63) else x


def _srl(z, k: int):
    """Logical right shift of int64 tensors."""
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(z, k), (1 << (64 - k)) - 1)


def _mix_t(z):
    """The SplitMix64 finaliser on int64 tensors (multiplications wrap modulo 2^64)."""
    import torch
    z = torch.bitwise_xor(z, _srl(z, 30)) * _to_i64(int(_M1))
    z = torch.bitwise_xor(z, _srl(z, 27)) * _to_i64(int(_M2))
    return torch.bitwise_xor(z, _srl(z, 31))


def uniform_t(seed: int, tag: int, start: int, count: int, device):
    """Device twin of uniform(): 53-bit uniforms in [0, 1), float64 tensor."""
    import torch
    s0 = _to_i64(int(stream_seed(seed, tag)))
    n = torch.arange(start + 1, start + 1 + count, dtype=torch.int64, device=device)
    z = _mix_t(s0 + n * _to_i64(int(_GOLDEN)))
    return _srl(z, 11).to(torch.float64) * 2.0 ** -53


def normal_t(seed: int, tag: int, start: int, count: int, device):
    """Device twin of normal() (uniforms 2n and 2n+1, Box-Muller cosine branch)."""
    import torch
    u = uniform_t(seed, tag, 2 * start, 2 * count, device)
    u1 = 1.0 - u[0::2]
    u2 = u[1::2]
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * torch.pi * u2)


def make_amplitudes_device(o: int, v: int, seed: int, device="cuda", Q: int | None = None):
    """make_amplitudes() drawn on a CUDA device: dict of float64 tensors eps, B, t1, t2."""
    import torch
    N = o + v
    if Q is None:
        Q = 3 * N
    eps_o = torch.sort(-1.5 + 1.2 * uniform_t(seed, TAG_EPS_OCC, 0, o, device)).values
    eps_v = torch.sort(0.1 + 2.9 * uniform_t(seed, TAG_EPS_VIR, 0, v, device)).values
    iu, ju = torch.triu_indices(N, N, device=device)
    npair = iu.numel()
    B = torch.empty((Q, N, N), dtype=torch.float64, device=device)
    step = max(1, (1 << 25) // max(npair, 1))
    for q0 in range(0, Q, step):
        q1 = min(Q, q0 + step)
        x = normal_t(seed, TAG_B, q0 * npair, (q1 - q0) * npair, device).reshape(q1 - q0, npair) * B_SIGMA
        x = torch.clamp(torch.round(x / B_GRID) * B_GRID, -B_CLIP, B_CLIP)
        B[q0:q1, iu, ju] = x
        B[q0:q1, ju, iu] = x
    t1 = (normal_t(seed, TAG_T1, 0, o * v, device) * T1_SIGMA).reshape(o, v)
    ov = o * v
    # upper triangle (I <= J) of the (i a) x (j b) matrix in row-major order of the triangle
    t2m = torch.empty((ov, ov), dtype=torch.float64, device=device)
    I, J = torch.triu_indices(ov, ov, device=device)
    base = I * ov - I * (I - 1) // 2                       # draws before row I
    idx = base + (J - I)
    total = ov * (ov + 1) // 2
    chunk = 1 << 25
    for c0 in range(0, total, chunk):
        c1 = min(total, c0 + chunk)
        x = normal_t(seed, TAG_T2, c0, c1 - c0, device) * T2_SIGMA
        sel = slice(c0, c1)                                # idx is increasing: positions c0..c1 of the triangle
        t2m[I[sel], J[sel]] = x
        t2m[J[sel], I[sel]] = x
    del I, J, base, idx
    t2 = t2m.reshape(o, v, o, v).permute(0, 2, 1, 3).contiguous()
    return {"o": o, "v": v, "eps": torch.cat([eps_o, eps_v]), "B": B, "t1": t1.contiguous(), "t2": t2}


def device_job_from_factor(amp: dict):
    """Integral blocks from a device-drawn job (make_amplitudes_device): dict as device_job()."""
    import torch
    o, v, B = amp["o"], amp["v"], amp["B"]
    Q = B.shape[0]
    Bov = B[:, :o, o:].reshape(Q, o * v)
    Bvv = B[:, o:, o:].reshape(Q, v * v)
    Boo = B[:, :o, :o].reshape(Q, o * o)
    ovvv = torch.empty((o, v, v, v), dtype=torch.float64, device=B.device)
    for i in range(o):
        ovvv[i] = (Bov.reshape(Q, o, v)[:, i, :].T @ Bvv).reshape(v, v, v)
    return dict(eps=amp["eps"], t1=amp["t1"], t2=amp["t2"], ovvv=ovvv,
                ovoo=(Bov.T @ Boo).reshape(o, v, o, o).contiguous(),
                ovov=(Bov.T @ Bov).reshape(o, v, o, v).contiguous())


# ---------------------------------------------------------------------------
# Device copies of a job (large workloads): the integral blocks are formed on
# the GPU with FP64 matrix products of the same DF factor.  Because every B
# value sits on a 2^-20 grid, each product sum is exact, so the device blocks
# are bit-identical to the host ones (tests check this on sampled slices).
# ---------------------------------------------------------------------------

def device_job(amp: Amplitudes, device="cuda"):
    """dict of device float64 tensors eps, t1, t2, ovvv, ovoo, ovov for one job."""
    import torch
    o, v, Q = amp.o, amp.v, amp.Q
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    Bov = f(amp.B[:, :o, o:]).reshape(Q, o * v)
    Bvv = f(amp.B[:, o:, o:]).reshape(Q, v * v)
    Boo = f(amp.B[:, :o, :o]).reshape(Q, o * o)
    ovvv = torch.empty((o, v, v, v), dtype=torch.float64, device=device)
    for i in range(o):
        ovvv[i] = (Bov.reshape(Q, o, v)[:, i, :].T @ Bvv).reshape(v, v, v)
    out = dict(eps=f(amp.eps), t1=f(amp.t1), t2=f(amp.t2), ovvv=ovvv,
               ovoo=(Bov.T @ Boo).reshape(o, v, o, o).contiguous(),
               ovov=(Bov.T @ Bov).reshape(o, v, o, v).contiguous())
    del Bov, Bvv, Boo
    return out
