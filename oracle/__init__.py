"""CPU oracle for the pseudo-stereo (DIBR) pipeline -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library (``paper_2009_09501_gb300``) never imports,
links or runs anything from here, and nothing here imports the product library.

Contents:
  dibr_oracle.c      -- single-threaded C99 statement of every pipeline step (FP64 where
                        floating point), each function citing the paper section it follows;
  inpaint2d_oracle.c -- the iterative 2-D block inpainting of the paper's Fig. 3 pseudo-code;
  oracle.py          -- ctypes wrapper over the compiled C oracle (numpy in, numpy out);
  naive.py           -- an independent pure-Python restatement (explicit loops, different
                        formulation) used to cross-check the C oracle on tiny images;
  build.py           -- compiles the C oracle with gcc.
"""
