"""CPU oracle for the block SRHT sketch and the low-rank algorithms built on it.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, FP64 restatement of
the paper (Balabanov, Beaupere, Grigori, Lederer, "Block subsampled randomized
Hadamard transform for low-rank approximation on distributed architectures"):

* ``philox``  - Philox4x64-10 counter-based generator (Salmon et al., SC'11),
                written from its published definition; the seeded signs and
                row samples of the block SRHT are drawn from it.
* ``bsrht``   - the Sylvester Hadamard matrix (tensor form, Sec. 2), the
                block SRHT Omega (eq. 2.3) as an explicit dense matrix, the
                sketch Omega A as a dense product (eq. 2.4), and a second,
                FWHT-based formulation used only to cross-check the first.
* ``lowrank`` - randomized SVD (Algorithm 1), randomized Nystrom
                (Algorithm 2 with Remark 3.1's shift) and the Eckart-Young
                optimum (Sec. 3), on numpy/LAPACK.
* ``gaussian``- the Gaussian embedding the paper compares against (Sec. 4),
                N(0, 1/l) entries from Philox and Box-Muller, and its sketch.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA library and never
imports it; the product path never calls into this package.
"""

from . import philox, bsrht, lowrank, gaussian  # noqa: F401
