"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws 4+4-bit offset-binary complex voltages with per-input noise
levels and injected RFI (a constant-phasor CW tone, or an on/off pulse), the
stand-in for CHIME's channelised F-engine output (paper Sec. 3.1, App. B: 4+4
bit complex Gaussian data bounded to [-7, 7]).  It contains none of the
detector's arithmetic.  The same bytes come out of the CPU generator
(`generate_cpu`) and the GPU generator (`generate_gpu`) for the same seed; see
`synth.h` for the sampler.

Workload recipes (seeded, synthetic):
  * `pathfinder_config`: 1 frequency, N=256, M=256, 64 frames, CW (A=3) in
    frames 10-19 and a period-32 pulse (A=4) in frames 40-44 (50 % duty by
    default, 25 % for the detectable variant).
  * `full_array_config`: F frequencies x N=2048, M=256, T frames; per
    frequency 2 % of frames carry CW and 1 % a 25 %-duty pulse, amplitudes
    U[1, 5].
  * `mixed_config`: frequencies of 2048 and 256 inputs with M drawn from
    {128, 256, 1024}.
Per-input sigma_i ~ U[1.5, 3.5] throughout.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CPU_LIB = os.path.join(HERE, "libsynth_cpu.so")
GPU_LIB = os.path.join(HERE, "libsynth_gpu.so")

NTHR = 14
TAG_PERM = 0x5045524D
TAG_AMP = 0x414D504C
BASE_SEED = 1808103650

_cpu = None
_gpu = None


def _load_cpu():
    global _cpu
    if _cpu is None:
        if not os.path.exists(CPU_LIB):
            from . import build as _b

            _b.build_cpu()
        lib = ctypes.CDLL(CPU_LIB)
        P = ctypes.c_void_p
        lib.synth_philox_block.argtypes = [P, P, P]
        lib.synth_u01.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_int64, P]
        lib.synth_sigmas.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_double, P]
        lib.synth_phases.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, P]
        lib.synth_thresholds.argtypes = [ctypes.c_double, ctypes.c_double, P]
        lib.synth_clean_tables.argtypes = [ctypes.c_int32, P, P]
        lib.synth_rfi_tables.argtypes = [ctypes.c_uint64, ctypes.c_int32, P, ctypes.c_int32,
                                         P, P, P]
        lib.synth_generate_cpu.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                           P, P, P]
        _cpu = lib
    return _cpu


def _load_gpu():
    global _gpu
    if _gpu is None:
        if not os.path.exists(GPU_LIB):
            raise RuntimeError(f"GPU generator library missing: {GPU_LIB} (run build())")
        lib = ctypes.CDLL(GPU_LIB)
        P = ctypes.c_void_p
        lib.synth_generate_gpu.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                           P, P, P, P]
        lib.synth_generate_gpu.restype = ctypes.c_int
        _gpu = lib
    return _gpu


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox_block(ctr, key) -> np.ndarray:
    """One Philox4x32-10 output block (4 words) for counter `ctr`, key `key`."""
    lib = _load_cpu()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib.synth_philox_block(_ptr(c), _ptr(k), _ptr(o))
    return o


def u01(seed: int, tag: int, a: int, b: int, n: int) -> np.ndarray:
    lib = _load_cpu()
    o = np.zeros(n, dtype=np.float64)
    lib.synth_u01(seed, tag, a, b, n, _ptr(o))
    return o


def sigmas(seed: int, N: int, lo: float = 1.5, hi: float = 3.5) -> np.ndarray:
    lib = _load_cpu()
    o = np.zeros(N, dtype=np.float64)
    lib.synth_sigmas(seed, N, lo, hi, _ptr(o))
    return o


def thresholds(sigma: float, shift: float = 0.0) -> np.ndarray:
    lib = _load_cpu()
    o = np.zeros(NTHR, dtype=np.uint32)
    lib.synth_thresholds(float(sigma), float(shift), _ptr(o))
    return o


def sub_seed(cfg: int, part: int, base: int = BASE_SEED) -> int:
    """Deterministic 64-bit seed of part `part` (a frequency or a stream) of workload `cfg`."""
    return (base + 0x9E3779B97F4A7C15 * (cfg * 65536 + part + 1)) % (1 << 64)


@dataclass
class RFI:
    frame: int          # frame index inside the dataset
    kind: str           # "cw" or "pulse"
    amp: float
    period: int = 1
    on_len: int = 1


@dataclass
class Dataset:
    """One frequency channel: n_frames frames of M samples for N inputs."""

    n_frames: int
    M: int
    N: int
    seed: int
    layout: int = 0                 # 0 time-major [frame][t][input]; 1 input-major
    sigma: Optional[np.ndarray] = None
    rfi: List[RFI] = field(default_factory=list)

    def __post_init__(self):
        if self.sigma is None:
            self.sigma = sigmas(self.seed, self.N)
        self.sigma = np.ascontiguousarray(self.sigma, dtype=np.float64)
        self._tables = None

    @property
    def frame_bytes(self) -> int:
        return self.M * self.N

    @property
    def nbytes(self) -> int:
        return self.n_frames * self.M * self.N

    def tables(self):
        """(thr_clean [N,14], frames [n_frames,4] int32, thr_rfi [slots,N,2,14])."""
        if self._tables is None:
            lib = _load_cpu()
            tc = np.zeros((self.N, NTHR), dtype=np.uint32)
            lib.synth_clean_tables(self.N, _ptr(self.sigma), _ptr(tc))
            fr = np.zeros((self.n_frames, 4), dtype=np.int32)
            fr[:, 0] = -1
            fr[:, 1] = 1
            fr[:, 2] = 1
            ns = len(self.rfi)
            slot_frame = np.array([r.frame for r in self.rfi], dtype=np.int64)
            slot_amp = np.array([r.amp for r in self.rfi], dtype=np.float64)
            tr = np.zeros((max(ns, 1), self.N, 2, NTHR), dtype=np.uint32)
            if ns:
                lib.synth_rfi_tables(self.seed, self.N, _ptr(self.sigma), ns,
                                     _ptr(slot_frame), _ptr(slot_amp), _ptr(tr))
            for s, r in enumerate(self.rfi):
                fr[r.frame] = (s, r.period, r.on_len, 0)
            self._tables = (tc, fr, tr)
        return self._tables

    def generate_cpu(self, frame0: int = 0, n: Optional[int] = None) -> np.ndarray:
        """Bytes of frames [frame0, frame0+n) as uint8 [n, M*N] (layout as set)."""
        if n is None:
            n = self.n_frames - frame0
        lib = _load_cpu()
        tc, fr, tr = self.tables()
        out = np.empty((n, self.M * self.N), dtype=np.uint8)
        frs = np.ascontiguousarray(fr[frame0:frame0 + n])
        lib.synth_generate_cpu(_ptr(out), n, frame0, self.M, self.N, self.layout, self.seed,
                               _ptr(tc), _ptr(frs), _ptr(tr))
        return out

    def generate_gpu(self, dst, frame0: int = 0, n: Optional[int] = None, stream=None):
        """Fill the uint8 CUDA tensor `dst` (>= n*M*N bytes) with frames [frame0, frame0+n)."""
        import torch

        if n is None:
            n = self.n_frames - frame0
        lib = _load_gpu()
        tc, fr, tr = self.tables()
        dev = dst.device
        d_tc = torch.from_numpy(tc.view(np.int32)).to(dev)
        d_fr = torch.from_numpy(np.ascontiguousarray(fr[frame0:frame0 + n])).to(dev)
        d_tr = torch.from_numpy(tr.view(np.int32)).to(dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        rc = lib.synth_generate_gpu(ctypes.c_void_p(dst.data_ptr()), n, frame0, self.M, self.N,
                                    self.layout, self.seed, ctypes.c_void_p(d_tc.data_ptr()),
                                    ctypes.c_void_p(d_fr.data_ptr()),
                                    ctypes.c_void_p(d_tr.data_ptr()),
                                    ctypes.c_void_p(s.cuda_stream))
        if rc != 0:
            raise RuntimeError("synth_generate_gpu failed")
        s.synchronize()


def pathfinder_config(seed: Optional[int] = None, duty: float = 0.5, N: int = 256, M: int = 256,
                      n_frames: int = 64) -> Dataset:
    """1 frequency, N=256, M=256, 64 frames; CW (A=3) frames 10-19, pulse (A=4, period 32) frames 40-44."""
    if seed is None:
        seed = sub_seed(0, 0)
    period = 32
    on = int(round(duty * period))
    rfi = [RFI(f, "cw", 3.0) for f in range(10, 20) if f < n_frames]
    rfi += [RFI(f, "pulse", 4.0, period, on) for f in range(40, 45) if f < n_frames]
    return Dataset(n_frames=n_frames, M=M, N=N, seed=seed, rfi=rfi)


def rfi_plan(seed: int, n_frames: int, cw_frac: float = 0.02, pulse_frac: float = 0.01,
             amp_lo: float = 1.0, amp_hi: float = 5.0, period: int = 32,
             pulse_duty: float = 0.25) -> List[RFI]:
    """Disjoint CW and pulse frames drawn by a seeded permutation; amplitudes U[amp_lo, amp_hi]."""
    n_cw = int(cw_frac * n_frames)
    n_pu = int(pulse_frac * n_frames)
    order = np.argsort(u01(seed, TAG_PERM, 0, 0, n_frames), kind="stable")
    amps = amp_lo + (amp_hi - amp_lo) * u01(seed, TAG_AMP, 0, 0, n_cw + n_pu)
    on = int(round(pulse_duty * period))
    out = [RFI(int(order[j]), "cw", float(amps[j])) for j in range(n_cw)]
    out += [RFI(int(order[n_cw + j]), "pulse", float(amps[n_cw + j]), period, on)
            for j in range(n_pu)]
    out.sort(key=lambda r: r.frame)
    return out


def full_array_config(n_freq: int = 4, n_frames: int = 1525, N: int = 2048, M: int = 256,
                      cfg: int = 1) -> List[Dataset]:
    """F frequencies x N inputs, M samples, T frames each; 2 % CW + 1 % pulse per frequency."""
    out = []
    for f in range(n_freq):
        s = sub_seed(cfg, f)
        out.append(Dataset(n_frames=n_frames, M=M, N=N, seed=s, rfi=rfi_plan(s, n_frames)))
    return out


def mixed_config(n_big: int = 64, n_small: int = 64, n_frames: int = 500,
                 Ms=(128, 256, 1024), cfg: int = 2) -> List[Dataset]:
    """Frequencies of 2048 inputs then of 256 inputs; M per frequency drawn from Ms by the seed."""
    out = []
    for f in range(n_big + n_small):
        s = sub_seed(cfg, f)
        N = 2048 if f < n_big else 256
        M = int(Ms[int(u01(s, TAG_AMP, 1, 0, 1)[0] * len(Ms))])
        out.append(Dataset(n_frames=n_frames, M=M, N=N, seed=s, rfi=rfi_plan(s, n_frames)))
    return out
