"""FP64 CPU oracle for the Relative Resolution (RelRes) Lennard-Jones path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may load it.  It is a plain, slow, obviously correct
restatement of Section 2 of Chaimovich & Chaimovich, "Relative Resolution: A
Computationally Efficient Implementation in LAMMPS" (arXiv:2104.10231):

* ``oracle.params``  -- FG mixing, the zero-order multipole sum rule (Eq. 13,
  Eq. 15), the per-site CG assignment (Eq. 14), the smoothing coefficients
  (Eq. 17, Eq. 18) and the shift constants (Eq. 19), all in FP64 Python.
* ``oracle/relres_oracle.c`` -- the literal five-region potential of Eq. 20
  summed over all atom pairs (O(N^2), minimum image), the bonded terms, and
  velocity-Verlet with a CSVR thermostat, in FP64 C.
* ``oracle.core`` -- ctypes wrapper around the C part.

It shares no code, header, table or constant with the CUDA path.  Parity for
every function here is pinned by ``tests/test_oracle_*.py`` (see the pin list
at the top of each test module).  Functions without an independent pin say
"parity unpinned" in their docstring.
"""
