"""GB300-native sparse inverse Cholesky factors of dense kernel matrices by greedy
conditional selection (Huan, Guinness, Katzfuss, Owhadi, Schaefer).

`sic` is the thin binding of the C-ABI library libsic (include/sic.h);
`pipeline` strings its calls into a whole factor build.
"""
from . import sic  # noqa: F401

__all__ = ["sic"]
