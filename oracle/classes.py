"""Quartet-class bookkeeping of arXiv 2303.13632 (test infrastructure).

Sec. II-A: shell size n_g = (L+1)(L+2)/2.
Sec. II-B, Eq. 3: canonical classes satisfy L_a >= L_b, L_c >= L_d and n_ga n_gb >= n_gc n_gd.
Sec. III-C: trip counts of the FPGA loops after the general optimisation
    n_RR = 3 n_Rys (L_d + 1), n_GQ = n_gc n_gd, n_CS = ceil(n_ERIQ / floor(512 / n)).
Sec. IV-B, Eq. 12: GERIS_model = f_max n_ERIQ / (max(n_RR, n_GQ, n_CS) + 10).
The Rys order is not printed; n_Rys = floor(L/2) + 1 with L = La+Lb+Lc+Ld is the
reading that reproduces every general-optimisation n_RR of Table III.
"""
from __future__ import annotations

import itertools
import math

SHELL_LETTERS = "spdf"


def n_g(L: int) -> int:
    return (L + 1) * (L + 2) // 2


def n_rys(La: int, Lb: int, Lc: int, Ld: int) -> int:
    return (La + Lb + Lc + Ld) // 2 + 1


def n_eriq(La: int, Lb: int, Lc: int, Ld: int) -> int:
    return n_g(La) * n_g(Lb) * n_g(Lc) * n_g(Ld)


def n_rr(La: int, Lb: int, Lc: int, Ld: int) -> int:
    return 3 * n_rys(La, Lb, Lc, Ld) * (Ld + 1)


def n_gq(La: int, Lb: int, Lc: int, Ld: int) -> int:
    return n_g(Lc) * n_g(Ld)


def n_cs(La: int, Lb: int, Lc: int, Ld: int, bits: int = 16) -> int:
    return math.ceil(n_eriq(La, Lb, Lc, Ld) / (512 // bits))


def geris_model(f_max_hz: float, n_eri: int, n_rr_: int, n_gq_: int, n_cs_: int) -> float:
    return f_max_hz * n_eri / (max(n_rr_, n_gq_, n_cs_) + 10) / 1e9


def is_canonical(La: int, Lb: int, Lc: int, Ld: int) -> bool:
    return La >= Lb and Lc >= Ld and n_g(La) * n_g(Lb) >= n_g(Lc) * n_g(Ld)


def all_classes(lmax: int = 3):
    return list(itertools.product(range(lmax + 1), repeat=4))


def class_name(La: int, Lb: int, Lc: int, Ld: int) -> str:
    s = SHELL_LETTERS
    return f"[{s[La]}{s[Lb]}|{s[Lc]}{s[Ld]}]"


def parse_class(name: str):
    t = name.strip("[]()").replace("|", "")
    return tuple(SHELL_LETTERS.index(ch) for ch in t)
