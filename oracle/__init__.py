"""CPU oracle for the amplitude path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct FP64 implementations of what the CUDA path
computes, written from the paper (Boixo, Isakov, Smelyanskiy, Neven,
"Simulation of low-depth quantum circuits as complex undirected graphical
models", arXiv:1712.05384):

* ``gates``        gate matrices from their definitions (Sec. "Numerical results")
* ``statevector``  the amplitude <x|C|0^n> as the product of the gate unitaries
                   (the definition behind Eq. fpath)
* ``pathsum``      brute-force Feynman path sum (Eq. fpath / Eq. psi_x) and the
                   exact Z[omega] Ising form (App. F, Eq. path1)
* ``ve``           bucket (variable) elimination on the complex graphical
                   model (Sec. III-IV, App. A) in its own vertical order
* ``order``        elimination orders and widths: fill-in simulation (Sec. IV.B),
                   vertical order (Sec. IV.A), min-fill, exact treewidth by
                   subset dynamic programming, line graph (App. E)
* ``xeb``          cross-entropy / Porter-Thomas statistics (App. B, C)

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import anything here.  Nothing here imports the CUDA package, and the
CUDA package never imports this one.  Parity status of each module is stated
in its header; every function is pinned by a ``-m "not gpu"`` test against
values fixed by the paper or by mathematics.
"""
