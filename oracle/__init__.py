"""Plain, slow FP64 CPU oracle of the nested single-layer CTMRG energy and gradient.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA path never imports it and shares no code with it; the two
meet only in the seeded inputs of ``workloads``.

Everything here is torch-CPU float64 and follows the paper step by step:

* ``nested``    - the nested single-layer network: ket A, bra A*, and the
                  virtual crossing tensors X and Y (Eq. XY), materialised as
                  explicit delta tensors; the reduced double-layer tensor
                  (Eq. Tred) for the cross-check.
* ``ctmrg``     - multisite CTMRG (Sec. SLF, Fig. 3): left move with projectors
                  from QR + SVD (Eqs. PQ, QRSVD), other moves by rotating the
                  network; reverse mode through a hand-written projector
                  adjoint (the SVD adjoint of the bond density matrix).
* ``energy``    - impurity reduced density matrices and Eq. ExpH.
* ``counter``   - multiply-add counts of every contraction and decomposition
                  (the algorithmic work of an evaluation).
* ``exact``     - finite clusters contracted without truncation, the exact
                  state vector and Lanczos ground state (used to pin the rest).

Readings of the paper where it is silent or garbled are listed, one by one, in
the module docstrings that make them.  Parity status of each function is given
in its docstring: all functions here are pinned by ``tests/test_oracle_*.py``.
"""
