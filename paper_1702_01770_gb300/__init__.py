"""GB300-native multicanonical (MUCA) sweep of off-lattice AB heteropolymers.

The hot path of PHAST (arXiv 1702.01770): many independent walkers, each making
pivot, crankshaft and rigid-chain moves scored by bending, torsion and
Lennard-Jones energy changes, accepted with tabulated multicanonical weights
and counted into energy histograms; around it Berg's weight recursion and the
microcanonical analysis.  The computation runs in hand-written CUDA kernels for
sm_103a behind the C ABI of ``include/phast.h`` (``libphast.so``); the Python
binding (``paper_1702_01770_gb300.phast``) only marshals arguments.

``paper_1702_01770_gb300.inputs`` builds the seeded synthetic workloads.
"""

__all__ = ["inputs", "phast"]
