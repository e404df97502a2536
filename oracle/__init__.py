"""CPU oracle for randomized Gram-Schmidt (RGS) and RGS-GMRES.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call, link or execute anything in this
package; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.

Two independent implementations live here:

* ``oracle.philox`` / ``oracle.sketch`` / ``oracle.rgs`` / ``oracle.gmres``:
  NumPy, FP64, written step by step from Balabanov & Grigori, "Randomized
  Gram-Schmidt process with application to GMRES" (Alg. 2, Alg. 3, Eq. hls);
* ``oracle/c/rgs_oracle.c``: plain C99, FP64 loops, the same algorithms with a
  hand-written incremental Householder least-squares solver
  (``oracle.c_oracle`` loads it with ctypes).

They share no code with each other beyond the published definitions they
both restate, and none with the GPU path.
"""
