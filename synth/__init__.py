"""Seeded synthetic self-heterodyne comb frames (arXiv 2307.12988, "Experimental Setup").

This module only *synthesises* inputs: RF interferogram frames of a comb whose
teeth sit at |51 MHz + k * 10 MHz| (the AOM offset and the EOM comb spacing of
the paper's setup), each tooth's amplitude shaped by the cavity resonance, plus
Gaussian noise, quantised to 12 bits in int16.  It holds none of the readout or
fitting arithmetic, and serves the oracle and the CUDA path alike.

Recipe (every number is a parameter; defaults follow the workloads):
  * tooth k: signed RF frequency f_k = 51 MHz + 10 MHz k, optical offset
    x_k = 10 MHz k (the fit abscissa);
  * per stream, drawn once: envelope e_k ~ U(0.9, 1.1) and phase
    phi_k ~ U[0, 2 pi), shared by the cavity and the reference frames, so the
    envelope cancels under normalisation;
  * per frame i with start time t_i = i N / fs: the cavity centre follows the
    mechanical drive, c_i = A_c sin(2 pi 23.686 kHz t_i) (the accelerometer's
    resonance); the lineshape is a Lorentzian dip
    L(x) = 1 - depth g^2 / ((x-c_i)^2 + g^2), g = FWHM / 2, or the literal
    peak g^2 / ((x-c_i)^2 + g^2); reference frames have L = 1;
  * sample n of frame i: sum_k E e_k L_i(x_k) cos(2 pi f_k (t_i + n/fs) + phi_k)
    with E = 512 sqrt(2/T), so the noise-free RMS is 1/4 of the 12-bit full
    scale (2048), plus N(0, sigma^2) noise; sigma is given directly or from a
    time-domain SNR, sigma = 512 / 10^(SNR/20);
  * quantisation: round half to even, clip to [-2048, 2047], store as int16.
Frames are generated in chunks of ``CHUNK`` frames, each chunk from its own
seed (stream seed, chunk index), so any frame can be regenerated alone.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FULL_SCALE = 2048.0          # 12-bit signed full scale
RMS_TARGET = 512.0           # noise-free RMS = FULL_SCALE / 4
AOM_OFFSET_HZ = 51e6         # LO shift by the acousto-optic modulator
COMB_SPACING_HZ = 10e6       # electro-optic comb spacing
DRIVE_HZ = 23.686e3          # mechanical resonance, used as the centre drive
FWHM_HZ = 80e6               # cavity linewidth (finesse 9200, length 203 um)
CHUNK = 4096
BASE_SEED = 2307_12988


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Digitiser rate, frame length and the comb teeth read out."""
    sample_rate: float
    frame_len: int
    k_lo: int
    k_hi: int

    @property
    def k(self) -> np.ndarray:
        return np.arange(self.k_lo, self.k_hi + 1)

    @property
    def n_teeth(self) -> int:
        return self.k_hi - self.k_lo + 1

    @property
    def tooth_freqs(self) -> np.ndarray:
        """Signed RF frequency of each tooth in Hz."""
        return AOM_OFFSET_HZ + COMB_SPACING_HZ * self.k.astype(np.float64)

    @property
    def tooth_x(self) -> np.ndarray:
        """Optical offset of each tooth in Hz (the fit abscissa)."""
        return COMB_SPACING_HZ * self.k.astype(np.float64)


# The workloads: 1 us frames at 1.0 / 1.1 / 2.5 GS/s (integer 1 MHz bins)
# and the 2.048 us, 2.0 GS/s serving stream whose teeth fall between bins.
TINY = Geometry(1.0e9, 1000, -10, 10)
PAPER_RATE = Geometry(1.1e9, 1100, -49, 49)
WIDE = Geometry(2.5e9, 2500, -110, 110)
SERVE_4096 = Geometry(2.0e9, 4096, -100, 100)
# the paper's digitiser frame: 8-bit samples at 2.2 GS/s, 2200 per 1 us row
PAPER_8BIT = Geometry(2.2e9, 2200, -49, 49)


@dataclasses.dataclass
class Stream:
    """Per-stream constants drawn once: tooth envelope and phases."""
    geom: Geometry
    envelope: np.ndarray
    phase: np.ndarray
    seed: int


def make_stream(geom: Geometry, seed: int) -> Stream:
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5EED]))
    env = rng.uniform(0.9, 1.1, geom.n_teeth)
    ph = rng.uniform(0.0, 2.0 * math.pi, geom.n_teeth)
    return Stream(geom, env, ph, seed)


def _cycles(f_hz: np.ndarray, num: np.ndarray, fs: float) -> np.ndarray:
    """Fractional cycles of f * num / fs, exact when f and fs are integral Hz."""
    f_int = np.rint(f_hz)
    if float(fs).is_integer() and np.all(f_int == f_hz):
        fsi = np.int64(fs)
        fr = np.mod(f_int.astype(np.int64), fsi)
        prod = np.mod(np.multiply.outer(fr, np.asarray(num, dtype=np.int64) % fsi), fsi)
        return prod.astype(np.float64) / float(fs)
    v = np.multiply.outer(f_hz, np.asarray(num, dtype=np.float64)) / fs
    return v - np.floor(v)


def lineshape(x: np.ndarray, c: np.ndarray, fwhm: np.ndarray | float,
              depth: np.ndarray | float = 0.7, shape: str = "dip", fano_q: float = 0.0) -> np.ndarray:
    """Cavity transmission factor per tooth, shape [n_frames, T].  "dip" and
    "peak" are Lorentzian; "fano" is the asymmetric profile
    (1 - depth) + depth (q + e)^2 / (1 + e^2), e = (x - c) / (fwhm / 2), whose
    baseline is 1 and whose q = 0 case is the dip."""
    g = np.asarray(fwhm, dtype=np.float64)[..., None] / 2.0 if np.ndim(fwhm) else fwhm / 2.0
    d = x[None, :] - np.asarray(c, dtype=np.float64)[:, None]
    dep = np.asarray(depth, dtype=np.float64)
    if dep.ndim:
        dep = dep[:, None]
    if shape == "fano":
        e = d / g
        return (1.0 - dep) + dep * (fano_q + e) ** 2 / (1.0 + e * e)
    lor = (g * g) / (d * d + g * g)
    if shape == "peak":
        return lor
    return 1.0 - dep * lor


def frames(stream: Stream, n_frames: int, *, first_frame: int = 0, cavity: bool = True,
           center_amp_hz: float = 5e6, drive_hz: float = DRIVE_HZ, fwhm_hz=FWHM_HZ,
           depth=0.7, shape: str = "dip", sigma=None,
           snr_db=None, noise_stream: int = 0, centers=None, device=None, bits: int = 12,
           fano_q: float = 0.0) -> dict:
    """Synthesise ``n_frames`` int16 frames [n_frames, N] (see the module recipe).

    ``centers`` (per frame, Hz) replaces the sinusoidal drive; ``fwhm_hz``,
    ``sigma`` and ``snr_db`` may be per-frame arrays.  ``device`` = None / "cpu"
    uses numpy; a torch CUDA device builds the frames there with torch (for the
    largest workloads).  ``bits`` = 12 (int16 storage) or 8 (int8, the paper's
    digitiser format): full scale 2^(bits-1), the noise-free RMS a quarter of
    it, the SNR-derived noise scaled with it (an explicit ``sigma`` is in
    output units).  Returns dict(frames, centers)."""
    g = stream.geom
    N, T, fs = g.frame_len, g.n_teeth, g.sample_rate
    if bits not in (8, 12):
        raise ValueError("bits must be 8 or 12")
    fs_full = 2.0 ** (bits - 1)
    rms = RMS_TARGET * fs_full / FULL_SCALE
    if sigma is None:
        sigma = 0.0 if snr_db is None else rms / 10.0 ** (np.asarray(snr_db, dtype=np.float64) / 20.0)
    sigma = np.asarray(sigma, dtype=np.float64)
    E = rms * math.sqrt(2.0 / T)
    idx = np.arange(first_frame, first_frame + n_frames, dtype=np.int64)
    t0 = idx.astype(np.float64) * N / fs
    if centers is None:
        centers = center_amp_hz * np.sin(2.0 * math.pi * drive_hz * t0)
    centers = np.asarray(centers, dtype=np.float64)
    if cavity:
        shape_f = lineshape(g.tooth_x, centers, fwhm_hz, depth, shape, fano_q)
    else:
        shape_f = np.ones((n_frames, T))
    amp = E * stream.envelope[None, :] * shape_f                    # [n, T]
    psi = 2.0 * math.pi * _cycles(g.tooth_freqs, idx * N, fs).T     # [n, T]
    theta = 2.0 * math.pi * _cycles(g.tooth_freqs, np.arange(N), fs) + stream.phase[:, None]
    Cb, Sb = np.cos(theta), np.sin(theta)                            # [T, N]
    ac, asn = amp * np.cos(psi), amp * np.sin(psi)
    if device is not None and str(device) != "cpu":
        out = _frames_torch(ac, asn, Cb, Sb, sigma, stream.seed, noise_stream,
                            first_frame, device, fs_full)
    else:
        out = np.empty((n_frames, N), dtype=np.int8 if bits == 8 else np.int16)
        for s in range(0, n_frames, CHUNK):
            e = min(n_frames, s + CHUNK)
            sig = ac[s:e] @ Cb - asn[s:e] @ Sb
            if np.any(sigma > 0):
                sg = sigma[s:e, None] if sigma.ndim else sigma
                sig += sg * _chunk_noise(stream.seed, noise_stream, first_frame + s, e - s, N)
            out[s:e] = np.clip(np.rint(sig), -fs_full, fs_full - 1).astype(out.dtype)
    return dict(frames=out, centers=centers)


def _chunk_noise(seed: int, noise_stream: int, first: int, n: int, N: int) -> np.ndarray:
    """Standard normals for frames [first, first+n); chunk-aligned seeding."""
    out = np.empty((n, N))
    i = 0
    while i < n:
        f = first + i
        chunk = f // CHUNK
        off = f - chunk * CHUNK
        take = min(n - i, CHUNK - off)
        rng = np.random.default_rng(np.random.SeedSequence([seed, 1 + noise_stream, chunk]))
        block = rng.standard_normal((off + take, N))
        out[i:i + take] = block[off:off + take]
        i += take
    return out


def _frames_torch(ac, asn, Cb, Sb, sigma, seed, noise_stream, first_frame, device, fs_full=FULL_SCALE):
    import torch
    dev = torch.device(device)
    n = ac.shape[0]
    N = Cb.shape[1]
    Ct = torch.from_numpy(Cb.astype(np.float32)).to(dev)
    St = torch.from_numpy(Sb.astype(np.float32)).to(dev)
    odt = torch.int8 if fs_full == 128.0 else torch.int16
    out = torch.empty((n, N), dtype=odt, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed((seed * 1_000_003 + noise_stream * 7919 + first_frame) % (2**63))
    step = 1 << 16
    for s in range(0, n, step):
        e = min(n, s + step)
        a1 = torch.from_numpy(ac[s:e].astype(np.float32)).to(dev)
        a2 = torch.from_numpy(asn[s:e].astype(np.float32)).to(dev)
        sig = a1 @ Ct - a2 @ St
        if np.any(sigma > 0):
            sg = (torch.from_numpy(sigma[s:e].astype(np.float32)).to(dev)[:, None] if sigma.ndim
                  else float(sigma))
            sig += sg * torch.randn(sig.shape, generator=gen, device=dev)
        out[s:e] = torch.clamp(torch.round(sig), -fs_full, fs_full - 1).to(odt)
    return out


def learned_params(n: int, *, seed: int, center_range_hz=100e6, fwhm_range_hz=(60e6, 100e6),
                   snr_range_db=(20.0, 40.0)) -> dict:
    """Per-frame cavity parameters of the learned-guess workload: centre
    U(-range, range), FWHM U(lo, hi), time-domain SNR U(lo, hi) dB."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x1EA4]))
    return dict(c=rng.uniform(-center_range_hz, center_range_hz, n),
                fwhm=rng.uniform(fwhm_range_hz[0], fwhm_range_hz[1], n),
                snr_db=rng.uniform(snr_range_db[0], snr_range_db[1], n))


def tooth_domain_spectra(geom: Geometry, n: int, *, seed: int, center_range_hz=100e6,
                         fwhm_range_hz=(60e6, 100e6), snr_range_db=(20.0, 40.0),
                         depth: float = 0.7) -> dict:
    """Normalised tooth spectra synthesised directly in the tooth domain.

    Each tooth's DFT value is the noise-free tooth phasor (amplitude E N/2 times
    the lineshape, random phase) plus complex Gaussian bin noise of standard
    deviation sigma sqrt(N/2) per component; y is its magnitude divided by the
    noise-free reference magnitude E N/2 (the envelope cancels).  Centres,
    linewidths and SNR are drawn per spectrum.  Returns dict(y, c, fwhm, snr_db)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x7D]))
    T, N = geom.n_teeth, geom.frame_len
    c = rng.uniform(-center_range_hz, center_range_hz, n)
    fwhm = rng.uniform(fwhm_range_hz[0], fwhm_range_hz[1], n)
    snr = rng.uniform(snr_range_db[0], snr_range_db[1], n)
    sigma = RMS_TARGET / 10.0 ** (snr / 20.0)
    E = RMS_TARGET * math.sqrt(2.0 / T)
    ref = E * N / 2.0
    shape_f = lineshape(geom.tooth_x, c, fwhm, depth, "dip")
    phase = rng.uniform(0.0, 2.0 * math.pi, (n, T))
    sb = (sigma * math.sqrt(N / 2.0) / ref)[:, None]
    re = shape_f * np.cos(phase) + sb * rng.standard_normal((n, T))
    im = shape_f * np.sin(phase) + sb * rng.standard_normal((n, T))
    y = np.sqrt(re * re + im * im)
    return dict(y=y, c=c, fwhm=fwhm, snr_db=snr)


def oscillator_series(n: int, fs: float, f0: float, Q: float, rms: float, floor: float = 0.0,
                      seed: int = 0) -> np.ndarray:
    """A thermally driven mechanical resonator sampled at fs: the AR(2)
    recursion x_i = 2 r cos(w_d) x_{i-1} - r^2 x_{i-2} + e_i of a damped
    oscillator (r = exp(-pi f0 / (Q fs)), w_d = 2 pi f0 / fs sqrt(1 - 1/4Q^2))
    driven by white noise, scaled to the given RMS, plus a white floor of
    standard deviation ``floor``; float64 [n]."""
    from scipy.signal import lfilter
    rng = np.random.default_rng(seed)
    r = math.exp(-math.pi * f0 / (Q * fs))
    wd = 2.0 * math.pi * f0 / fs * math.sqrt(1.0 - 1.0 / (4.0 * Q * Q))
    burn = int(20 * Q * fs / f0) + 16                 # let the recursion forget its zero start
    e = rng.standard_normal(n + burn)
    x = lfilter([1.0], [1.0, -2.0 * r * math.cos(wd), r * r], e)[burn:]
    x *= rms / np.std(x)
    if floor:
        x += floor * rng.standard_normal(n)
    return x
