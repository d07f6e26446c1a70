"""CPU FP64 oracle for the MPS-ANO-VQC feature-extraction path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` use it.  It shares no code with the
CUDA path: the two meet only in ``paper_2607_10280_b300.synth`` (seeded input
generators, which hold none of the method's arithmetic).

Modules, each a plain restatement of the paper:

* ``circuit``     gate matrices and the ordered gate lists of the two ansaetze
                  (Sec. II.B, Eq. 2; the benchmark ansatz with trainable-free
                  R_Y/R_Z rotations and an ascending CNOT ladder).
* ``statevector`` dense 2^n simulator (n <= 20) and the definition
                  <psi| P_a (x) P_b |psi> (Sec. II.C, Eq. 5).
* ``mps``         matrix-product-state simulator with SVD truncation to bond
                  chi at the orthogonality centre (Sec. II.B, Eq. 3) and
                  environment contraction of the pair Paulis (Eq. 5).
* ``pairs``       image-local pair lists (Sec. II.C).
* ``ano``         Hermitian observables from (A, B, D), Pauli coefficients
                  c = 2^-2 Tr(H P) (Eq. 4), features (Eq. 5) and the linear
                  reconstruction layer (Eq. 6).
* ``train``       training on cached Paulis (Sec. II.C-D): MSE term of Eq. 7,
                  its gradients by the chain rule, and the two Adam optimizers.

Pins: every function here is checked by ``tests/test_oracle_*.py`` and
``tests/test_train_oracle.py`` against
values fixed by the paper or by mathematics (closed forms, brute-force
Kronecker products, Clifford conjugation, Schmidt truncation of the dense
state, Pauli-basis completeness).  No function is "parity unpinned".
"""
