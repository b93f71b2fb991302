"""Seeded synthetic inputs: WDM pulse trains and dispersion-managed fiber maps.

This module builds the inputs that both the CUDA path and the CPU oracle
consume.  It holds none of the propagation arithmetic: it only describes the
fiber (a list of piecewise-constant segments repeated periodically, the loss
and the amplifier spacing of Eq. (1)) and draws a time-domain field A(t) on a
periodic grid t_n = n*T/N from a seeded PCG64 generator.

Units follow Eq. (1): t in ps, z in km, beta2 in ps^2/km, beta3 in ps^3/km,
sigma in 1/(W km), |A|^2 in W.  gamma is the amplitude loss coefficient of
Eq. (1) (G = -gamma between amplifiers), so a power loss of a dB/km is
gamma = a*ln(10)/20 per km, and the amplifier gain exp(z_a*gamma) restores
exactly the span loss.

The paper's own system parameters live in a cited 2002 letter that is not
available, so the named workloads below are synthetic stand-ins with the
channel counts, symbol counts, pulse shapes and DM map of the configurations
this library is benchmarked on.
"""
from __future__ import annotations

import dataclasses
import json
import math
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "Segment",
    "FiberMap",
    "Workload",
    "gamma_from_db_per_km",
    "wdm_field",
    "dm_map",
    "workload",
    "load_workload",
    "save_workload",
    "WORKLOADS",
]


@dataclasses.dataclass(frozen=True)
class Segment:
    """One piece of the DM period with constant coefficients (Eq. (1))."""

    length_km: float
    beta2_ps2_per_km: float
    beta3_ps3_per_km: float
    sigma_per_W_km: float
    gain_per_km: float = 0.0  # distributed amplitude gain g: G = g - gamma between amplifiers


@dataclasses.dataclass(frozen=True)
class FiberMap:
    """Periodic DM fiber: ``segments`` form one period, repeated ``n_periods`` times.

    Lumped amplifiers sit at z_k = k * z_a_km (k >= 1) and multiply the field by
    exp(z_a * gamma) (the delta-function part of G(z) in Eq. (1)).
    """

    segments: Tuple[Segment, ...]
    gamma_per_km: float
    z_a_km: float
    n_periods: int

    @property
    def period_km(self) -> float:
        return float(sum(s.length_km for s in self.segments))

    @property
    def length_km(self) -> float:
        return self.period_km * self.n_periods

    def as_rows(self) -> np.ndarray:
        """Segments as an (n, 5) float64 array: length, beta2, beta3, sigma, gain."""
        return np.array(
            [[s.length_km, s.beta2_ps2_per_km, s.beta3_ps3_per_km, s.sigma_per_W_km, s.gain_per_km]
             for s in self.segments],
            dtype=np.float64,
        )


def gamma_from_db_per_km(db_per_km: float) -> float:
    """Amplitude loss coefficient for a power loss given in dB/km."""
    return db_per_km * math.log(10.0) / 20.0


def dm_map(
    n_periods: int,
    beta3: float = 0.1,
    sigma: float = 1.3,
    loss_db_per_km: float = 0.2,
    d1: Tuple[float, float] = (45.0, -21.7),
    d2: Tuple[float, float] = (5.0, 190.0),
) -> FiberMap:
    """The two-segment DM span of the benchmark links: 45 km of anomalous fiber,
    5 km of compensating fiber, then a lumped amplifier every 50 km."""
    segs = (
        Segment(d1[0], d1[1], beta3, sigma),
        Segment(d2[0], d2[1], beta3, sigma),
    )
    return FiberMap(segs, gamma_from_db_per_km(loss_db_per_km), d1[0] + d2[0], n_periods)


def wdm_field(
    N: int,
    T_ps: float,
    n_channels: int,
    spacing_GHz: float,
    n_symbols: int,
    fwhm_ps: float,
    peak_mW: float,
    modulation: str,
    seed: int,
) -> np.ndarray:
    """Seeded WDM pulse train on the periodic grid t_n = n*T/N (complex128).

    Each channel c carries one return-to-zero Gaussian pulse per symbol slot of
    width T/n_symbols, intensity FWHM ``fwhm_ps`` and peak power ``peak_mW``.
    ``modulation`` is "ook" (bit 0 = no pulse, Bernoulli(1/2)) or "qpsk" (pulse
    always present, phase uniform in {0, pi/2, pi, 3pi/2}).  Channel c sits at
    the frequency offset f_c = (c - (n_channels-1)/2) * spacing; with the
    Fourier convention A_hat = int A exp(+i w t) dt it is written as
    exp(-2 pi i f_c t) so that it appears at +w_c.  Every offset is a whole
    number of grid frequencies 1/T for the named workloads, so the field is
    exactly periodic.
    """
    if N % n_symbols != 0:
        raise ValueError("N must be a multiple of the symbol count")
    rng = np.random.Generator(np.random.PCG64(seed))
    spp = N // n_symbols  # samples per slot
    slot = T_ps / n_symbols
    dt = T_ps / N
    t0 = fwhm_ps / (2.0 * math.sqrt(math.log(2.0)))  # |A|^2 = P0 exp(-t^2/t0^2)
    amp0 = math.sqrt(peak_mW * 1e-3)
    # pulse centred in its slot; neighbours out to +-3 slots (tails < 1e-30 for the named widths)
    tl = (np.arange(spp) + 0.0) * dt - 0.5 * slot
    reach = 3
    shapes = [np.exp(-((tl + d * slot) ** 2) / (2.0 * t0 * t0)) for d in range(-reach, reach + 1)]
    t = np.arange(N, dtype=np.float64) * dt
    field = np.zeros(N, dtype=np.complex128)
    for c in range(n_channels):
        if modulation == "ook":
            sym = rng.integers(0, 2, size=n_symbols).astype(np.complex128)
        elif modulation == "qpsk":
            sym = np.exp(0.5j * math.pi * rng.integers(0, 4, size=n_symbols))
        else:
            raise ValueError(f"unknown modulation {modulation!r}")
        train = np.zeros((n_symbols, spp), dtype=np.complex128)
        for i, d in enumerate(range(-reach, reach + 1)):
            # slot s holds the tail of the pulse of symbol s-d, whose centre is
            # d slots earlier (periodic wrap: np.roll(sym, d)[s] = sym[s-d])
            train += np.roll(sym, d)[:, None] * shapes[i][None, :]
        fc = (c - 0.5 * (n_channels - 1)) * spacing_GHz * 1e-3  # THz = 1/ps
        cycles = fc * T_ps
        if abs(cycles - round(cycles)) > 1e-9:
            raise ValueError("channel offset is not a whole number of grid frequencies")
        field += amp0 * train.reshape(N) * np.exp(-2j * math.pi * fc * t)
    return field


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named link: input field recipe, fiber map and the method settings."""

    name: str
    N: int
    T_ps: float
    n_channels: int
    spacing_GHz: float
    n_symbols: int
    fwhm_ps: float
    peak_mW: float
    modulation: str
    seed: int
    fiber: FiberMap
    ss_dz_km: float
    mpa_L_km: float
    mpa_M: int
    mpa_n_iter: int

    def field(self) -> np.ndarray:
        return wdm_field(self.N, self.T_ps, self.n_channels, self.spacing_GHz, self.n_symbols,
                         self.fwhm_ps, self.peak_mW, self.modulation, self.seed)

    @property
    def length_km(self) -> float:
        return self.fiber.length_km

    def to_dict(self) -> dict:
        """Plain-JSON form (the fiber map as its segment list)."""
        d = dataclasses.asdict(self)
        d["fiber"]["segments"] = [dataclasses.asdict(seg) for seg in self.fiber.segments]
        return d

    @classmethod
    def from_dict(cls, d: dict) -> "Workload":
        """Inverse of :meth:`to_dict`; a "note" key is allowed and ignored,
        any other unknown or missing key is an error."""
        d = {k: v for k, v in d.items() if k != "note"}
        names = {f.name for f in dataclasses.fields(cls)}
        if set(d) != names:
            raise ValueError(f"workload keys: missing {sorted(names - set(d))}, unknown {sorted(set(d) - names)}")
        fd = dict(d["fiber"])
        segs = tuple(Segment(**seg) for seg in fd.pop("segments"))
        fiber = FiberMap(segs, float(fd.pop("gamma_per_km")), float(fd.pop("z_a_km")), int(fd.pop("n_periods")))
        if fd:
            raise ValueError(f"unknown fiber keys {sorted(fd)}")
        ints = {"N", "n_channels", "n_symbols", "seed", "mpa_M", "mpa_n_iter"}
        kw = {k: (int(v) if k in ints else v if k in ("name", "modulation") else float(v))
              for k, v in d.items() if k != "fiber"}
        return cls(fiber=fiber, **kw)


def load_workload(path: str) -> Workload:
    """Workload from a JSON file written by :func:`save_workload` (or by hand
    in the same form)."""
    with open(path) as f:
        return Workload.from_dict(json.load(f))


def save_workload(w: Workload, path: str, note: str = "") -> None:
    d = w.to_dict()
    if note:
        d = {"note": note, **d}
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")


def _wl0() -> Workload:
    # 4 ch @ 50 GHz, 128 OOK bits at 10 Gb/s, 30 ps FWHM, 1 mW, N=2^14, 4 spans (200 km);
    # MPA: L = 50 km (one span), M = 800 (dz = 0.0625 km, a node on the 45-km
    # jump), n_tot = 3.  Over the first two spans against FP64 split-steps at
    # dz/8, dz/16 (Richardson, uncertainty 5e-8) the split-step at dz = 0.1 km
    # errs 5.21e-5 and the MPA at M = 710, 750, 800, 850 5.54e-5, 5.93e-5,
    # 4.94e-5, 3.50e-5 (n_tot = 4 changes nothing: the quadrature dominates;
    # L = 25 km with M = 400 and L = 10 km with M = 160 give the same 4.94e-5)
    return Workload("wdm4_ook_n2p14_200km", 1 << 14, 12800.0, 4, 50.0, 128, 30.0, 1.0, "ook", 0,
                    dm_map(4), 0.1, 50.0, 800, 3)


def _wl1() -> Workload:
    # 16 ch @ 50 GHz, 1024 QPSK symbols, 30 ps FWHM, 2 mW, N=2^20, 40 spans (2000 km);
    # MPA: L = 5 km, n_tot = 2, M = 125 (dz = 0.04 km): the equal-accuracy
    # choice over the first two spans against a FP64 split-step at dz/4, dz/8
    # with Richardson (SS at dz = 0.05 km: 1.00e-2; MPA n_tot = 2 at M = 100,
    # 110, 120, 130, 142: 1.06e-2, 1.03e-2, 9.8e-3, 8.5e-3, 7.2e-3; reference
    # uncertainty 2.5e-4), so the coarsest M that stays below the split-step's
    # error with a margin of several reference uncertainties
    return Workload("wdm16_qpsk_n2p20_2000km", 1 << 20, 102400.0, 16, 50.0, 1024, 30.0, 2.0, "qpsk", 1,
                    dm_map(40), 0.05, 5.0, 125, 2)


def _wl2() -> Workload:
    # 64 ch @ 25 GHz, 2048 QPSK symbols at 10 GBd, N=2^24, beta3=0.08, 100 spans (5000 km);
    # MPA: L = 5 km, M = 142, n_tot = 4.  Over the first two spans against FP64
    # split-steps at dz/4, dz/8 (Richardson) the split-step at dz = 0.05 km
    # errs 6.7e-2 and the MPA at n_tot = 3 1.04e-1 whatever M (142, 213, 284:
    # 1.04e-1, 9.9e-2, 9.6e-2: the Picard iteration, contraction about 0.43 on
    # this 64-channel link, dominates), at n_tot = 4 5.5e-2
    return Workload("wdm64_qpsk_n2p24_5000km", 1 << 24, 204800.0, 64, 25.0, 2048, 30.0, 2.0, "qpsk", 2,
                    dm_map(100, beta3=0.08), 0.05, 5.0, 142, 4)


def _wl4() -> Workload:
    # gradients: 16 ch @ 50 GHz, 512 QPSK symbols per channel in 100 ps slots,
    # N=2^20, 20 spans (1000 km); the method settings of the 2^20 link
    return Workload("wdm16_qpsk512_n2p20_1000km", 1 << 20, 51200.0, 16, 50.0, 512, 30.0, 2.0, "qpsk", 4,
                    dm_map(20), 0.05, 5.0, 142, 2)


WORKLOADS = {"0": _wl0, "1": _wl1, "2": _wl2, "4": _wl4}


def workload(key: str) -> Workload:
    """Named workload by index ("0", "1", "2", "4"), by name, or from a JSON
    file (a path ending in ".json", see :func:`load_workload`)."""
    if key.endswith(".json"):
        return load_workload(key)
    if key in WORKLOADS:
        return WORKLOADS[key]()
    for f in WORKLOADS.values():
        w = f()
        if w.name == key:
            return w
    raise KeyError(key)


def random_field(N: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Small seeded complex test field with standard-normal parts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal(N) + 1j * rng.standard_normal(N)) * scale


def chirped_gaussian(N: int, T_ps: float, t0_ps: float, peak_mW: float, chirp: float = 0.0,
                     centre_ps: float | None = None) -> np.ndarray:
    """sqrt(P0) exp(-(1 + i C) (t - tc)^2 / (2 t0^2)) on the periodic grid
    (nearest periodic image of the centre)."""
    t = np.arange(N, dtype=np.float64) * (T_ps / N)
    tc = 0.5 * T_ps if centre_ps is None else centre_ps
    d = (t - tc + 0.5 * T_ps) % T_ps - 0.5 * T_ps
    return math.sqrt(peak_mW * 1e-3) * np.exp(-(1.0 + 1j * chirp) * d * d / (2.0 * t0_ps * t0_ps))


@dataclasses.dataclass(frozen=True)
class LinkSpec:
    """One link of a batch: its own window, channels, power, sigma and length."""

    N: int
    T_ps: float
    n_channels: int
    peak_mW: float
    sigma: float
    spans: int
    seed: int

    @property
    def fiber(self) -> FiberMap:
        return dm_map(self.spans, sigma=self.sigma)

    @property
    def length_km(self) -> float:
        return 50.0 * self.spans

    def field(self) -> np.ndarray:
        # slots of 100 ps sampled at 256 points: the 16-channel comb (+-375 GHz)
        # stays well inside the +-1.28 THz band of the grid
        return wdm_field(self.N, self.T_ps, self.n_channels, 50.0, self.N // 256, 30.0, self.peak_mW, "qpsk",
                         self.seed)


def batch_links(n_links: int = 256, seed: int = 3, log2_n=(12, 18), spans=(1, 20)) -> List[LinkSpec]:
    """Seeded batch of independent links: N uniform in 2^12..2^18, channel
    count in {2, 4, 8, 16}, 1-20 DM spans, sigma uniform in [1.0, 1.6] /W/km,
    launch (peak) power uniform in [0.5, 4] mW; all on the benchmark DM map."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_links):
        logn = int(rng.integers(log2_n[0], log2_n[1] + 1))
        N = 1 << logn
        out.append(LinkSpec(N=N, T_ps=100.0 * (N // 256), n_channels=int(rng.choice([2, 4, 8, 16])),
                            peak_mW=float(rng.uniform(0.5, 4.0)), sigma=float(rng.uniform(1.0, 1.6)),
                            spans=int(rng.integers(spans[0], spans[1] + 1)), seed=1000 + i))
    return out
