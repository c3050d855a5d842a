"""FP64 CPU oracle of the coherent F-statistic (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The library under
``paper_0904_1826_gb300`` never imports it and shares no code with it.

Pinned functions (see tests/test_oracle_pins.py):
  * detector kinematics, timing, antenna patterns  -- closed forms, finite
    differences, the JKS antenna formulas;
  * some_calculations / compute_fa_fb / normalized -- brute-force
    time-domain demodulation, the noise-free closed form, the chi^2_4 noise law;
  * toplist                                        -- exhaustive sort on ties;
  * quantisation                                   -- exactly representable cases;
  * the MLP forward/backward                       -- central finite differences;
  * noise floor, whitening, noise weights           -- closed-form medians and weights,
    stationary invariance, chi^2_4 mean on non-stationary noise;
  * c_oracle (the same F-statistic as plain C loops, for whole workunits)
    -- equality with the numpy oracle, the noise-free closed form and its
    D -> infinity limit, planted mistakes (tests/test_oracle_c.py).
"""
from . import fstat_oracle  # noqa: F401
from . import mlp_oracle  # noqa: F401
from . import noise_oracle  # noqa: F401
from . import quantize  # noqa: F401
