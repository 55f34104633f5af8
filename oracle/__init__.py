"""Independent FP64 CPU oracle for the lattice Boltzmann scheme for the
Kuramoto-Sivashinsky equation (Otomo, Boghosian & Dubois, arXiv:1711.03540).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library.

Modules
-------
lbks        ctypes front end of ``lbks_oracle.c`` (the LB scheme itself, FP64,
            periodic or front-test reservoir boundaries).
analysis    linear amplification matrix of one LB step, growth rates,
            truncation-error predictions of Sec. 2.2, stability scans.
spectral    pseudo-spectral ETDRK4 solver of the KS equation (Kassam &
            Trefethen, SIAM J. Sci. Comput. 26 (2005)), an independent
            reference for convergence checks.
front       the analytic travelling-front solution of Table 5 and the global
            relative error G of Sec. 3.
"""
