"""CPU FP64 oracle for the preconditioned iPEPS hot path (test infrastructure).

This package is a plain, slow, obviously-correct restatement of what the
method computes, written from the paper: CTMRG environments (Sec. III.A),
the nearest-neighbour energy (Eq. equ:energy), its gradient at the CTMRG
fixed point, the local-metric preconditioner (Eq. equ:local_metric) with the
delta regularisation (Sec. III.B) and the GMRES(30) solve (Sec. III.C), and
plain / preconditioned L-BFGS (Sec. II, Sec. IV.A).

It is test infrastructure only: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with the CUDA path; the only common module is the seeded input generator.

Parity-pin status per function is listed in each module's header.
"""
