"""FP64 CPU oracle of the PRC-LBM (arXiv:2208.03562).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_2208_03562_gb300`` and never imports it.

* ``oracle.stepper``   -- ctypes front end of ``prc_oracle.c``: the step list of
  Appendix A, literally, in FP64 (oracle-A).
* ``oracle.matrix_form`` -- the single-node collision as the matrix product of
  Eq. 10-equivalent-centralmoment with the main-text coefficients of
  Eqs. 38-48 (oracle-B), in numpy.
"""
