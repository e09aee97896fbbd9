"""CPU oracle for the spheroidal boundary-integral-operator apply.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 (complex128
for oblate spheroids) restatement of the method of "Boundary integral equation
analysis for spheroidal suspensions" (Crowder, Li, Corona, Veerapaneni): the
spheroidal coordinates of Sec. 2.1, the off-the-cut Legendre algorithm of
Sec. 2.3, the layer-potential theorems of Sec. 3 (Theorems 1 and 2), the
near/far splitting and smooth quadrature of Sec. 4 (Algorithm 1) and the
Laplace-to-Stokes identity of Sec. 4.3.

It shares no code with the CUDA library and imports nothing from it.  Only the
test-suite, the smoke check and the CPU-baseline leg of the benchmark may
import it; the product path never does.

Modules
    legendre   P_n^m / Q_n^m off the cut (real x > 1 or x = i u), Ferrers
               functions on the cut and the real surface-harmonic basis
    geometry   spheroid parameters, quadrature nodes, coordinate inversion,
               point-to-spheroid distance, near sets
    laplace    Theorem 1/2 multipliers, self / exterior / interior evaluation,
               far-field quadrature and the two apply modes
               (O-method: what the GPU computes; O-exact: no quadrature error)
    stokes     Laplace-to-Stokes single layer (Sec. 4.3)
    brute      oversampled direct quadrature used only to pin the above
"""
