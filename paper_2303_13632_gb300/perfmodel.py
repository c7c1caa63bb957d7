"""Algorithmic work per quartet class: the numerator of each kernel's roofline.

FLOPs are counted like arXiv 2303.13632 counts n_FLOPQ (Sec. III-A: add, multiply and
divide count one each, an FMA two), per primitive quartet of the canonical class the kernel
evaluates:
  setup       40 + 20 n_Rys     Gaussian-product prefactors (40, FP64) and the B, C arrays
                                (20 n_Rys: FP64 on the plain path; on the mixed path FP32 in
                                two-float arithmetic where the class uses that setup, see
                                two_float_setup, else FP64)
  roots       60 n_Rys          Rys roots/weights (done on the host in the paper) (FP64 on the
                                plain path; 20 n_Rys FP64 + 40 n_Rys R on the mixed path)
  VRR         5 * 3 n_Rys * ((La+Lb+1)(Lc+Ld+1) - 1)                            (R)
  HRR         2 per produced entry of the bra and ket transfers                 (R)
  quadrature  3 n_Rys n_ERIQ                                                     (R)
  compress    2 n_ERIQ + 1                                                       (R)
R is FP64 on the plain path and FP32 on the mixed path.  Bytes per quartet: 16 in (four
int32 shell ids; shell data is cache resident) and n_ERIQ * bits / 8 + 4 out (compressed) or
8 n_ERIQ out (FP64).

Default peaks (GB300, 152 SMs at the 2070 MHz maximum clock): FP32 = 152 x 128 lanes x 2 x
2.07 GHz = 80.5 TFLOP/s; FP64 = 1.25 TFLOP/s (the nominal figure for this part); the benchmark
passes the FMA rates it measures instead.  A kernel with F64 FP64 flops and F32 FP32 flops per
quartet needs at least F64/P64 + F32/P32 seconds per quartet on the ALUs and bytes/BW on HBM;
its roofline time is the larger of the two.
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


def two_float_setup(cls) -> bool:
    """Whether the mixed path forms the B, C arrays of class cls in two-float FP32 (the split
    setup kernel of every class not on the inline-setup thread-per-quartet kernel, and those
    inline kernels with two or more roots except [ds|ds] and [dp|ss])."""
    c = canonical(cls)
    n = sum(c) // 2 + 1
    if kernel_form(c) != "tpq_inline":
        return True
    return n >= 2 and c not in ((2, 0, 2, 0), (2, 1, 0, 0))


def flops_per_quartet(cls, precision: str = "fp64"):
    """(fp64_flops, rr_flops) per primitive quartet of class cls.  The root/weight evaluation
    (60 n) is FP64 on the plain path; the mixed path evaluates the polynomial terms beyond the
    fourth (and the Taylor terms of F_0/F_1 beyond the second) in FP32, a third / two thirds
    split of the same 60 n, counted 20 n FP64 + 40 n in the recurrence type.  The B, C arrays
    (20 n) count in the recurrence type where the mixed path forms them in two-float FP32."""
    La, Lb, Lc, Ld = canonical(cls)
    n = (La + Lb + Lc + Ld) // 2 + 1
    nab, ncd = La + Lb, Lc + Ld
    neri = ncart(La) * ncart(Lb) * ncart(Lc) * ncart(Ld)
    roots64 = 60 * n if precision == "fp64" else 20 * n
    bc64 = 0 if precision != "fp64" and two_float_setup(cls) else 20 * n
    f64 = 40 + bc64 + roots64
    vrr = 5 * 3 * n * ((nab + 1) * (ncd + 1) - 1)
    hrr_bra = sum((nab - j + 1) * (ncd + 1) for j in range(1, Lb + 1))
    hrr_ket = (La + 1) * (Lb + 1) * sum(ncd - l + 1 for l in range(1, Ld + 1))
    hrr = 2 * 3 * n * (hrr_bra + hrr_ket)
    quad = 3 * n * neri
    comp = 2 * neri + 1
    return f64, vrr + hrr + quad + comp + (60 * n - roots64) + (20 * n - bc64)


def adjoint_flops_per_quartet(cls, precision: str = "fp64"):
    """(fp64_flops, rr_flops) of the adjoint (eri_backward) per primitive quartet of class cls,
    counted like flops_per_quartet:
      setup       40 + 20 n' + 60 n'   geometry, B and C, roots on the extended class (every L + 2,
                                       n' = floor((L + 2) / 2) + 1 roots): FP64, except two thirds
                                       of the roots (40 n') in the recurrence type on the mixed
                                       path; the adjoint forms B and C in FP64 on both paths
      recurrences VRR + HRR of the extended class, as in flops_per_quartet              (R)
      contraction 3 flops (a multiply and an FMA) per root, axis and output: W = sum G I_y I_z
                  over the outputs sharing their x-components                           (R)
      derivative  30 per root, axis and tuple of x-components (w): four centres x (2 alpha
                  I(a+1) - a I(a-1), times W, accumulated: 5; W I(a+2) subtracted: 2), and the
                  exponent term W I (2)                                                 (R)
      finish      20 per quartet: the exponent gradients and the centre sums            (FP64)"""
    La, Lb, Lc, Ld = canonical(cls)
    n = (La + Lb + Lc + Ld + 2) // 2 + 1
    neri = ncart(La) * ncart(Lb) * ncart(Lc) * ncart(Ld)
    wn = (La + 1) * (Lb + 1) * (Lc + 1) * (Ld + 1)
    ea, eb, ec, ed = La + 2, Lb + 2, Lc + 2, Ld + 2
    nab, ncd = ea + eb, ec + ed
    vrr = 5 * 3 * n * ((nab + 1) * (ncd + 1) - 1)
    hrr_bra = sum((nab - j + 1) * (ncd + 1) for j in range(1, eb + 1))
    hrr_ket = (ea + 1) * (eb + 1) * sum(ncd - l + 1 for l in range(1, ed + 1))
    hrr = 2 * 3 * n * (hrr_bra + hrr_ket)
    contraction = 3 * 3 * n * neri
    derivative = 30 * 3 * n * wn
    roots64 = 60 * n if precision == "fp64" else 20 * n
    f64 = 40 + 20 * n + roots64 + 20
    return f64, vrr + hrr + contraction + derivative + (60 * n - roots64)


def bytes_per_quartet(cls, bits: int) -> int:
    neri = ncart(cls[0]) * ncart(cls[1]) * ncart(cls[2]) * ncart(cls[3])
    out = neri * 8 if bits == 0 else (neri * bits + 7) // 8 + 4
    return 16 + out


def roofline_seconds(cls, n_quartets: int, precision: str, bits: int, hbm_gbs: float,
                     p32: float = PEAK_FP32_TFLOPS, p64: float = PEAK_FP64_TFLOPS) -> float:
    """Shortest time for n_quartets quartets of class cls: the slower of the ALU time (FP64 flops
    at the FP64 peak plus FP32 flops at the FP32 peak, TFLOP/s) and the HBM time."""
    f64, rr = flops_per_quartet(cls, precision)
    if precision == "fp64":
        t_alu = (f64 + rr) / (p64 * 1e12)
    else:
        t_alu = f64 / (p64 * 1e12) + rr / (p32 * 1e12)
    t_mem = bytes_per_quartet(cls, bits) / (hbm_gbs * 1e9)
    return n_quartets * max(t_alu, t_mem)


def fp32_equivalent_flops(cls, precision: str, p32: float = PEAK_FP32_TFLOPS,
                          p64: float = PEAK_FP64_TFLOPS) -> float:
    """Work of one quartet expressed in FP32-pipe flops (FP64 flops weighted by the peak
    ratio), so that one number and one peak describe a mixed kernel."""
    f64, rr = flops_per_quartet(cls, precision)
    w = p32 / p64
    return f64 * w + (rr * w if precision == "fp64" else rr)


# ---------------------------------------------------------------------------------------------
# GPU analogue of the paper's throughput model (Eq. 12: f_max n_ERIQ / (max(n_RR, n_GQ, n_CS) +
# 10), the slowest pipelined stage plus a fixed per-quartet overhead).  On the GPU the FP64 setup
# and the FP32 recurrences/quadrature do not overlap as FPGA pipeline stages do: the split path
# runs them as two kernels one after the other, and in the inline form they share the warp
# schedulers.  So their times add, and the output bytes bound the sum from below; each stage runs
# at an effective rate, plus a per-quartet overhead that depends on the kernel form:
#     t_q = max(F64 / R64 + F32 / R32, B / BW) + o_form
# The rates and overheads are fitted to measured per-class times.

def kernel_form(cls) -> str:
    """The kernel form a primitive FP32 class runs in (inline-setup thread-per-quartet, split
    setup + FP32 thread-per-quartet, split setup + shared-memory phase kernel)."""
    La, Lb, Lc, Ld = canonical(cls)
    neri = ncart(La) * ncart(Lb) * ncart(Lc) * ncart(Ld)
    iblk = (La + 1) * (Lb + 1) * (Lc + 1) * (Ld + 1)
    if neri <= 36 and iblk <= 16:
        return "tpq_inline"
    if neri <= 100 and iblk <= 16:
        return "tpq_split"
    return "phase_split"


FORMS = ("tpq_inline", "tpq_split", "phase_split")


def model_seconds_per_quartet(cls, params, bits: int = 16) -> float:
    f64, rr = flops_per_quartet(cls, "mixed")
    t = max(f64 / params["R64"] + rr / params["R32"], bytes_per_quartet(cls, bits) / params["BW"])
    return t + params["o_" + kernel_form(cls)]


def fit_gpu_model(measured, bits: int = 16):
    """Fits R64, R32 (FLOP/s), BW (B/s) and one overhead per kernel form (s) to measured
    {class tuple: seconds per quartet}, minimising the squared log error."""
    import numpy as np
    from scipy.optimize import minimize

    classes = list(measured)
    t_meas = np.array([measured[c] for c in classes])

    def unpack(x):
        p = {"R64": np.exp(x[0]), "R32": np.exp(x[1]), "BW": np.exp(x[2])}
        for i, f in enumerate(FORMS):
            p["o_" + f] = np.exp(x[3 + i])
        return p

    def loss(x):
        p = unpack(x)
        t = np.array([model_seconds_per_quartet(c, p, bits) for c in classes])
        return float(np.sum(np.log(t / t_meas) ** 2))

    x0 = np.log([PEAK_FP64_TFLOPS * 1e12, PEAK_FP32_TFLOPS * 1e12, 5e12, 1e-12, 1e-12, 1e-12])
    res = minimize(loss, x0, method="Nelder-Mead", options={"maxiter": 20000, "maxfev": 20000,
                                                             "xatol": 1e-6, "fatol": 1e-9})
    p = unpack(res.x)
    t_fit = np.array([model_seconds_per_quartet(c, p, bits) for c in classes])
    err = np.log(t_fit / t_meas)
    return p, {"median_abs_log_err": float(np.median(np.abs(err))),
               "max_abs_log_err": float(np.max(np.abs(err))),
               "r2_log": float(1 - np.sum(err ** 2) / np.sum((np.log(t_meas) - np.mean(np.log(t_meas))) ** 2))}


def read_class_table(path):
    """{class tuple: (quartets, GERIS mixed)} from the committed per-class sweep table."""
    letters = {"s": 0, "p": 1, "d": 2, "f": 3}
    out = {}
    with open(path) as f:
        for line in f:
            if not line.startswith("| ["):
                continue
            name, rest = line[3:].split("] |", 1)  # "[ab\\|cd] | n | geris | ..."
            cells = [c.strip() for c in rest.strip().strip("|").split("|")]
            cls = tuple(letters[ch] for ch in name if ch in letters)
            out[cls] = (int(cells[0]), float(cells[1]))
    return out


if __name__ == "__main__":
    import sys

    table = read_class_table(sys.argv[1])
    measured = {c: ncart(c[0]) * ncart(c[1]) * ncart(c[2]) * ncart(c[3]) / (g * 1e9)
                for c, (n, g) in table.items()}
    p, q = fit_gpu_model(measured)
    print(f"R64 = {p['R64'] / 1e12:.3f} TFLOP/s, R32 = {p['R32'] / 1e12:.2f} TFLOP/s, "
          f"BW = {p['BW'] / 1e9:.0f} GB/s; per-quartet overheads: "
          + ", ".join(f"{f} {p['o_' + f] * 1e12:.1f} ps" for f in FORMS))
    print(f"median |log(t_model / t_measured)| = {q['median_abs_log_err']:.3f}, "
          f"max = {q['max_abs_log_err']:.3f}, R^2 (log t) = {q['r2_log']:.3f}")
