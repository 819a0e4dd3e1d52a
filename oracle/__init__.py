"""FP64 CPU oracle for the 2LPT f(R) displacement path (Moretti et al. 2019).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the method in float64 numpy, written to check the CUDA path.
Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference
leg of `bench.py` may import it.  It shares no code with the CUDA library
and never imports it; the two meet only in the seeded inputs of `workloads`.

Modules
  fft        own radix-2 FFT (plain DFT matrix for non power-of-two axes)
  philox     Philox4x32-10 counter-based generator + Box-Muller noise
  cosmology  background, Hu-Sawicki m^2(a), M2(a), mu(k,a), EH no-wiggle P(k)
  growth     RK4 growth tables D1(k,a), D2(k,a) (T1 triangle) and tangents
  lpt2       the pipeline: delta(k), Psi1, phi_ij, source, Psi2, CIC, P(k)
  vjp        hand adjoint of the pipeline

Every function states the passage of the paper (section / equation) it follows.
Readings of passages the paper leaves open are stated where they are used.
"""
