"""Plain, slow FP64 CPU oracle for the FC-SDNN Runge-Kutta stage (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library: it has its own FC-Gram
table builder (mpmath, 40 digits), its own FFT-based derivative (numpy FFT as a
library primitive), its own Euler operator, time stepping, patch exchange,
shock-detecting network, artificial viscosity and reductions.  The only module
both sides use is ``paper_2506_19370_gb300.inputs``, which builds seeded
initial data and patch layouts and holds none of the method's arithmetic.

Modules:
  fcgram  - FC-Gram continuation tables and FC derivatives (paper §2)
  euler   - Euler operator, boundary conditions, RK stages, exchange, Δt, sums
            (Eq. 1-3, §3.3, §5 items 1 and 4, Algorithms 1 and 5)
  sdnn    - proxy, windows, classifier MLP (forward, backward, Adam),
            coefficient-decay indicator, artificial viscosity (§4, §5 item 2,
            Algorithm 3)
  exact   - closed forms used as pins: exact Riemann solver, isentropic
            vortex, Mach-M shock states, oblique-shock relation (§7)
"""
