"""FP64 CPU oracle for the neural directed-distance-field (DDF) hot path.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct restatement
of what the CUDA path computes, written from the paper (arXiv 2306.16142) in float64
numpy. Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import it. The product library never calls it,
and it shares no code with the CUDA sources: the two meet only in the seeded input
generators of ``ddf_synth``.

Modules and the passages they follow:

* ``philox``  - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC'11), used by the renderer's draws.
* ``mlp``     - the DDF network MLP_w(x, theta) of Sec. 4.1 (forward), its input gradient
  for the surface normal of Eq. 3 / Sec. 4.2, its parameter gradient and the training
  loss, and the Adam update named in Sec. 5.1.
* ``label``   - ray labelling by nearest ray-triangle hit against the mesh (Sec. 1 /
  Sec. 6 "shot rays and calculated t"): brute-force Moeller-Trumbore over all faces.
* ``sphere``  - the analytic DDF of a sphere (closed form for the definitions of Sec. 3.1).
* ``render``  - the modified uni-directional path tracer (Sec. 1, Fig. 1): camera rays,
  one DDF query per bounce, Lambertian shading with cosine-hemisphere sampling; the same
  tracer's query with a mesh in place of the field (Fig. 5's comparison), and the depth and
  normal images of Fig. 3 / Fig. 4.
* ``udf``     - the unsigned distance field of Eq. 4 as a minimum over a direction set.
* ``sampler`` - the surface-marching training-set sampler of Sec. 5.2 (Eqs. 8-12) with the
  odd-even inside test, and the point-of-view and random sampling of Sec. 6, built on ``label``.
* ``head``    - the paper's single-output head with the clamp loss of Eq. 7 or the squish
  loss of Eq. 5, and the weight-normalised hidden layers of Sec. 5.1.

Every floating-point step runs in float64 from the float32 inputs (promoted exactly).
Where the paper is silent, the readings used are listed in each module's docstring.
"""
