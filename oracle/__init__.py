"""Plain FP64 CPU oracle for the iPEPS real-time evolution of the dilated disordered lattice.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct reference that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path (the C-ABI library and
its Python binding) never imports, links or calls anything here, and nothing here imports the
product package: the two share no code.  The only shared module is ``inputs/``, the seeded input
generators, which hold none of the method's arithmetic.

What the oracle computes (all complex128 / float64, LAPACK via NumPy for SVD and eigh):

* ``model``   -- local operators of the dilated site (hard-core boson x auxiliary spin-1/2), the
  bond Hamiltonian and its Trotter gate (Sec. "Set up for iPEPS", Eq. Hanc, written in
  hard-core-boson form), the CDW (x) |+> initial product state (Sec. "Set up for iPEPS",
  Initialization; Fig. 1).
* ``su``      -- the simple update of Jiang, Weng & Xiang (PRL 101, 090603 (2008)), cited by the
  paper for the quench (Sec. "Set up for iPEPS", Quench; Appendix), applied with the plain
  (unreduced) two-site tensor and a full SVD, first- and second-order Trotter sequences.
* ``ctmrg``   -- directional corner-transfer-matrix renormalisation (Orus & Vidal, PRB 80, 094403
  (2009); Orus, PRB 85, 205117 (2012)), cited by the paper for the readout (Sec. "Set up for
  iPEPS", Readout; Appendix), with the full 2x2-block projectors of Corboz, Rice & Troyer
  (PRL 113, 046402 (2014)), an explicit double-layer tensor and full SVDs.
* ``measure`` -- one- and two-site reduced density matrices from the converged environment, the
  disorder-averaged particle numbers, imbalance I = n_A - n_B (Sec. "Results for interacting
  case"), aux polarisation, energy per site and the CTM norm per site.
* ``evolve``  -- the time-evolution driver that alternates Trotter steps with CTMRG + measurement.

Parity status of each function is listed in its docstring.  The only unpinned piece is the
comparison with the paper's own curves: its figures carry no data.
"""
