"""Seeded synthetic channelised voltages for the X-engine.

This module only draws and packs input samples; it holds none of the
correlator's arithmetic.  Tests feed the same bytes to the CUDA path and to
the oracle.  Recipes (the shapes and value models of the Tianlai workloads):

* ``gauss``: re and im i.i.d. N(0, sigma^2), rounded half-to-even and clipped
  to [-clip, clip].  sigma = 2.5, clip = 7 mimics the 4-bit equaliser output
  whose RMS sits between 2 and 3 of the +-7 range (Sec. 2.1, F-engine,
  Eq. 3 and the equaliser text); sigma = 20, clip = 127 is the 8-bit case.
* ``sky``: a common sky signal plus independent receiver noise,
  x_i(c,t) = Q(amp * s(c,t) * exp(j phi_i(c)) + n_i(c,t)), with s complex
  Gaussian of unit power, n_i re/im ~ N(0, noise^2), and a per-input
  geometric phase phi_i(c) = 2 pi tau_i c / C + phi0_i that is linear in
  frequency -- the delay model of the paper's cable test (Sec. 3, Eq. 5).
  tau_i is an integer in [-C/8, C/8], phi0_i uniform in [0, 2 pi).

Packing: a 4-bit complex sample is one byte of two 4-bit two's-complement
numbers (Sec. 2.1: "two 4 bit real numbers are then re-packed to a 8-bit
complex number"); real in the high nibble unless ``hi_is_real`` is False.
An 8-bit sample is two int8 bytes (re, im).  Layouts: 0 = [t][c][i] (the
payload order of Sec. 2.3), 1 = [t][i][c], 2 = [c][i][t].
"""
from __future__ import annotations

import numpy as np

L_TCI, L_TIC, L_CIT = 0, 1, 2


def _quantise(v: np.ndarray, clip: int) -> np.ndarray:
    return np.clip(np.rint(v), -clip, clip).astype(np.int8)


def gauss(seed: int, n_inputs: int, n_chans: int, n_time: int, sigma: float = 2.5, clip: int = 7):
    """re, im int8 arrays [C][N][T] of i.i.d. quantised Gaussian samples."""
    rng = np.random.default_rng(seed)
    shape = (n_chans, n_inputs, n_time)
    re = _quantise(rng.standard_normal(shape, dtype=np.float32) * sigma, clip)
    im = _quantise(rng.standard_normal(shape, dtype=np.float32) * sigma, clip)
    return re, im


def sky_params(seed: int, n_inputs: int, n_chans: int):
    """Per-input integer delays tau_i and phase offsets phi0_i of the sky model."""
    rng = np.random.default_rng([seed, 7])
    lim = max(n_chans // 8, 0)
    tau = rng.integers(-lim, lim + 1, size=n_inputs)
    phi0 = rng.uniform(0.0, 2 * np.pi, size=n_inputs)
    return tau, phi0


def sky(seed: int, n_inputs: int, n_chans: int, n_time: int, amp: float = 0.5,
        noise: float = 1.0, clip: int = 7):
    """re, im int8 arrays [C][N][T] of the common-sky-plus-noise model."""
    rng = np.random.default_rng(seed)
    tau, phi0 = sky_params(seed, n_inputs, n_chans)
    c = np.arange(n_chans)[:, None]
    phase = 2 * np.pi * tau[None, :] * c / n_chans + phi0[None, :]  # [C][N]
    rot = np.exp(1j * phase).astype(np.complex64)
    s = (rng.standard_normal((n_chans, 1, n_time), dtype=np.float32)
         + 1j * rng.standard_normal((n_chans, 1, n_time), dtype=np.float32)) * np.float32(np.sqrt(0.5))
    x = amp * s * rot[:, :, None]
    x = x + noise * (rng.standard_normal((n_chans, n_inputs, n_time), dtype=np.float32)
                     + 1j * rng.standard_normal((n_chans, n_inputs, n_time), dtype=np.float32))
    return _quantise(x.real, clip), _quantise(x.imag, clip)


def to_layout(a: np.ndarray, layout: int) -> np.ndarray:
    """Reorder a canonical [C][N][T] array into the given sample order."""
    if layout == L_TCI:
        return np.ascontiguousarray(a.transpose(2, 0, 1))
    if layout == L_TIC:
        return np.ascontiguousarray(a.transpose(2, 1, 0))
    if layout == L_CIT:
        return np.ascontiguousarray(a)
    raise ValueError("unknown layout %r" % layout)


def pack(re: np.ndarray, im: np.ndarray, bits: int = 4, layout: int = L_TCI,
         hi_is_real: bool = True) -> np.ndarray:
    """Pack canonical [C][N][T] int samples into a flat uint8 block."""
    re = to_layout(np.asarray(re), layout)
    im = to_layout(np.asarray(im), layout)
    if bits == 4:
        r = re.astype(np.uint8) & 0xF
        m = im.astype(np.uint8) & 0xF
        hi, lo = (r, m) if hi_is_real else (m, r)
        return ((hi << 4) | lo).astype(np.uint8).reshape(-1)
    if bits == 8:
        out = np.empty(re.shape + (2,), dtype=np.int8)
        out[..., 0] = re
        out[..., 1] = im
        return out.view(np.uint8).reshape(-1)
    raise ValueError("bits must be 4 or 8")


def block(kind: str, seed: int, n_inputs: int, n_chans: int, n_time: int, bits: int = 4,
          layout: int = L_TCI, hi_is_real: bool = True, **kw) -> np.ndarray:
    """One packed block of a named recipe ("gauss" or "sky")."""
    clip = 7 if bits == 4 else 127
    if kind == "gauss":
        sigma = kw.get("sigma", 2.5 if bits == 4 else 20.0)
        re, im = gauss(seed, n_inputs, n_chans, n_time, sigma=sigma, clip=clip)
    elif kind == "sky":
        re, im = sky(seed, n_inputs, n_chans, n_time, amp=kw.get("amp", 0.5),
                     noise=kw.get("noise", 1.0), clip=clip)
    else:
        raise ValueError("unknown recipe %r" % kind)
    return pack(re, im, bits=bits, layout=layout, hi_is_real=hi_is_real)


def random_bytes(seed: int, nbytes: int) -> np.ndarray:
    """Uniform random bytes (every 4-bit code, including -8, equally likely)."""
    return np.random.default_rng(seed).integers(0, 256, size=nbytes, dtype=np.uint8)


def block_device(kind: str, seed: int, n_inputs: int, n_chans: int, n_time: int, layout: int,
                 device, bits: int = 4, chunk_time: int = 256):
    """The same recipes generated with torch directly in device memory.

    For workloads too large to draw on the host in reasonable time.  The
    values follow the same distributions as :func:`block` (not the same
    bytes); parity against the oracle then uses the bytes copied back.
    Layout 1 ([t][i][c]) and 0 ([t][c][i]) are produced time chunk by time
    chunk so that temporaries stay small.
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    clip = 7 if bits == 4 else 127
    N, C, T = n_inputs, n_chans, n_time
    bps = bits // 4
    out = torch.empty(N * C * T * bps, dtype=torch.uint8, device=device)
    if kind == "sky":
        tau, phi0 = sky_params(seed, N, C)
        cc = torch.arange(C, device=device, dtype=torch.float32)
        phase = (2 * np.pi * torch.as_tensor(tau, device=device, dtype=torch.float32)[:, None] * cc[None, :] / C
                 + torch.as_tensor(phi0, device=device, dtype=torch.float32)[:, None])  # [N][C]
        rot_re, rot_im = torch.cos(phase), torch.sin(phase)
    sigma = 2.5 if bits == 4 else 20.0
    if layout == L_CIT:
        chunk_time = T  # canonical [C][N][T]: generate per channel chunk instead
    for t0 in range(0, T, chunk_time):
        tn = min(chunk_time, T - t0)
        if kind == "gauss":
            re = torch.randn((tn, N, C), generator=g, device=device) * sigma
            im = torch.randn((tn, N, C), generator=g, device=device) * sigma
        else:
            s_re = torch.randn((tn, 1, C), generator=g, device=device) * np.sqrt(0.5)
            s_im = torch.randn((tn, 1, C), generator=g, device=device) * np.sqrt(0.5)
            re = 0.5 * (s_re * rot_re - s_im * rot_im) + torch.randn((tn, N, C), generator=g, device=device)
            im = 0.5 * (s_re * rot_im + s_im * rot_re) + torch.randn((tn, N, C), generator=g, device=device)
        re = torch.clamp(torch.round(re), -clip, clip).to(torch.int8)  # [t][i][c]
        im = torch.clamp(torch.round(im), -clip, clip).to(torch.int8)
        if layout == L_TCI:
            re = re.permute(0, 2, 1)
            im = im.permute(0, 2, 1)
        elif layout == L_CIT:
            re = re.permute(2, 1, 0)
            im = im.permute(2, 1, 0)
        if bits == 4:
            byte = ((re.to(torch.uint8) & 0xF) << 4) | (im.to(torch.uint8) & 0xF)
            flat = byte.contiguous().reshape(-1)
        else:
            flat = torch.stack([re, im], dim=-1).contiguous().view(torch.uint8).reshape(-1)
        if layout == L_CIT:
            out.copy_(flat)
        else:
            n = tn * N * C * bps
            out[t0 * N * C * bps: t0 * N * C * bps + n].copy_(flat)
    return out


def adc(seed: int, n_inputs: int, n_samples: int, sigma: float = 16.0, tones=(),
        common: float = 0.0) -> np.ndarray:
    """Seeded 8-bit ADC streams for the F-engine, int8 [n_inputs][n_samples].

    Each input is receiver noise N(0, sigma^2) plus, when ``common`` > 0, a
    noise signal N(0, common^2) shared by every input delayed by i samples
    (a broadband sky source seen through cables of different lengths, as in
    the paper's delay test, Sec. 3), plus the listed tones: (amplitude,
    cycles per sample, phase) added to every input.  Rounded half-to-even and
    clipped to the 8-bit range [-127, 127] of the digitiser.
    """
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, sigma, (n_inputs, n_samples))
    if common > 0:
        s = rng.normal(0.0, common, n_samples + n_inputs)
        for i in range(n_inputs):
            v[i] += s[n_inputs - i:n_inputs - i + n_samples]
    n = np.arange(n_samples, dtype=np.float64)
    for amp, f, ph in tones:
        v += amp * np.cos(2 * np.pi * f * n + ph)[None, :]
    return np.clip(np.rint(v), -127, 127).astype(np.int8)


def packets(block: np.ndarray, n_fids: int, n_inputs_pkt: int, n_xids: int, n_chans_pkt: int,
            block_index: int = 0) -> list:
    """Cut a [T][C][N] block of packed 4-bit samples into the F-engine's UDP
    payloads (Sec. 2.3): an 8-byte header (MCNT big-endian in 6 bytes, Fid,
    Xid), 8 stacked spectra of n_chans_pkt x n_inputs_pkt bytes, and an
    8-byte trailer (4 zero bytes, then the CRC-32 of header and payload from
    zlib, big-endian).  Packets come out MCNT by MCNT, Fid-major."""
    arr = packets_array(block, n_fids, n_inputs_pkt, n_xids, n_chans_pkt, block_index)
    return [row.tobytes() for row in arr]


def packets_array(block: np.ndarray, n_fids: int, n_inputs_pkt: int, n_xids: int,
                  n_chans_pkt: int, block_index: int = 0) -> np.ndarray:
    """The packets of :func:`packets` as one uint8 array [n_packets][length]."""
    import zlib
    T = block.shape[0]
    per = T // 8
    P = 8 * n_chans_pkt * n_inputs_pkt
    # [slot][8][xid][c][fid][i] -> [slot][fid][xid][8][c][i]
    pay = block.reshape(per, 8, n_xids, n_chans_pkt, n_fids, n_inputs_pkt).transpose(0, 4, 2, 1, 3, 5)
    n = per * n_fids * n_xids
    arr = np.zeros((n, 8 + P + 8), dtype=np.uint8)
    arr[:, 8:8 + P] = pay.reshape(n, P)
    slot, fid, xid = np.meshgrid(np.arange(per), np.arange(n_fids), np.arange(n_xids), indexing="ij")
    mcnt = (block_index * per + slot.reshape(-1)).astype(np.uint64)
    for k in range(6):
        arr[:, k] = ((mcnt >> np.uint64(8 * (5 - k))) & np.uint64(0xFF)).astype(np.uint8)
    arr[:, 6] = fid.reshape(-1)
    arr[:, 7] = xid.reshape(-1)
    for r in range(n):
        c = zlib.crc32(arr[r, :8 + P]) & 0xFFFFFFFF
        arr[r, 8 + P + 4:] = np.frombuffer(c.to_bytes(4, "big"), dtype=np.uint8)
    return arr
