"""Algorithmic work per quartet class: the numerator of each kernel's roofline.

FLOPs are counted like arXiv 2303.13632 counts n_FLOPQ (Sec. III-A: add, multiply and
divide count one each, an FMA two), per primitive quartet of the canonical class the kernel
evaluates:
  setup       40 + 20 n_Rys     Gaussian-product prefactors and B, C arrays       (FP64)
  roots       60 n_Rys          Rys roots/weights (done on the host in the paper) (FP64)
  VRR         5 * 3 n_Rys * ((La+Lb+1)(Lc+Ld+1) - 1)                            (R)
  HRR         2 per produced entry of the bra and ket transfers                 (R)
  quadrature  3 n_Rys n_ERIQ                                                     (R)
  compress    2 n_ERIQ + 1                                                       (R)
R is FP64 on the plain path and FP32 on the mixed path.  Bytes per quartet: 16 in (four
int32 shell ids; shell data is cache resident) and n_ERIQ * bits / 8 + 4 out (compressed) or
8 n_ERIQ out (FP64).

Peaks (GB300, 152 SMs at the 2070 MHz maximum clock): FP32 = 152 x 128 lanes x 2 x 2.07 GHz
= 80.5 TFLOP/s; FP64 = 1.25 TFLOP/s (the nominal figure for this part).  A kernel with F64
FP64 flops and F32 FP32 flops per quartet needs at least F64/P64 + F32/P32 seconds per
quartet on the ALUs and bytes/BW on HBM; its roofline time is the larger of the two.
"""
from __future__ import annotations

PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 1.25


def ncart(L: int) -> int:
    return (L + 1) * (L + 2) // 2


def canonical(cls):
    """Canonical representative (Sec. II-B, Eq. 3) of a generic class (La, Lb, Lc, Ld)."""
    La, Lb, Lc, Ld = cls
    bra = (La, Lb) if La >= Lb else (Lb, La)
    ket = (Lc, Ld) if Lc >= Ld else (Ld, Lc)
    if ncart(bra[0]) * ncart(bra[1]) < ncart(ket[0]) * ncart(ket[1]):
        bra, ket = ket, bra
    return bra + ket


def flops_per_quartet(cls):
    """(fp64_flops, rr_flops) per primitive quartet of class cls."""
    La, Lb, Lc, Ld = canonical(cls)
    n = (La + Lb + Lc + Ld) // 2 + 1
    nab, ncd = La + Lb, Lc + Ld
    neri = ncart(La) * ncart(Lb) * ncart(Lc) * ncart(Ld)
    f64 = 40 + 20 * n + 60 * n
    vrr = 5 * 3 * n * ((nab + 1) * (ncd + 1) - 1)
    hrr_bra = sum((nab - j + 1) * (ncd + 1) for j in range(1, Lb + 1))
    hrr_ket = (La + 1) * (Lb + 1) * sum(ncd - l + 1 for l in range(1, Ld + 1))
    hrr = 2 * 3 * n * (hrr_bra + hrr_ket)
    quad = 3 * n * neri
    comp = 2 * neri + 1
    return f64, vrr + hrr + quad + comp


def bytes_per_quartet(cls, bits: int) -> int:
    neri = ncart(cls[0]) * ncart(cls[1]) * ncart(cls[2]) * ncart(cls[3])
    out = neri * 8 if bits == 0 else (neri * bits + 7) // 8 + 4
    return 16 + out


def roofline_seconds(cls, n_quartets: int, precision: str, bits: int, hbm_gbs: float) -> float:
    f64, rr = flops_per_quartet(cls)
    if precision == "fp64":
        t_alu = (f64 + rr) / (PEAK_FP64_TFLOPS * 1e12)
    else:
        t_alu = f64 / (PEAK_FP64_TFLOPS * 1e12) + rr / (PEAK_FP32_TFLOPS * 1e12)
    t_mem = bytes_per_quartet(cls, bits) / (hbm_gbs * 1e9)
    return n_quartets * max(t_alu, t_mem)


def fp32_equivalent_flops(cls, precision: str) -> float:
    """Work of one quartet expressed in FP32-pipe flops (FP64 flops weighted by the peak
    ratio), so that one number and one peak describe a mixed kernel."""
    f64, rr = flops_per_quartet(cls)
    w = PEAK_FP32_TFLOPS / PEAK_FP64_TFLOPS
    return f64 * w + (rr * w if precision == "fp64" else rr)
