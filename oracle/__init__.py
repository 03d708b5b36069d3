"""Oracle: a plain, slow, float64 CPU implementation of the tree-level |M|^2.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package entry point's
smoke() check and the CPU-baseline leg of bench.py may import anything here.
The GPU product path never imports, links or calls this package, and this
package imports nothing from the GPU product path (it shares only the seeded
input generators in `phasespace`).

What it computes (method of arXiv:2503.21935, Sec. 2-3: event-parallel matrix
elements; Feynman diagrams in double precision followed by the colour-matrix
quadratic form and the helicity sum):

  me = 1/(4 * Ncol_in * S) * sum_h sum_colours | sum_terms A_t(h) c_t(colours) |^2

with A_t the Lorentz part of each Feynman-diagram term written out as an
explicit tensor contraction of external wavefunctions, vertex tensors and
propagators (textbook Feynman rules, Peskin & Schroeder conventions), and c_t the
explicit SU(3) colour tensor of that term.  The paper prints no formulas; the
rules follow HELAS (Murayama, Watanabe, Hagiwara, KEK-91-11) conventions for the
external states and the SM Feynman rules for vertices and propagators.

Pins (tests/test_oracle_*.py): closed forms (e+e- -> mu+mu- per helicity,
gg -> t tbar, gg -> gg), Lorentz invariance, gauge invariance, alpha_s scaling,
Bose symmetry, an independent Berends-Giele recursion, brute-force explicit
colour sums, exact colour-matrix entries and the diagram counts.
"""
