"""FP64 CPU oracle for the dG spherical-harmonic VFP operator of arXiv:2501.05110.

TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously-correct restatement of the paper's method:
spherical-harmonic coupling matrices by sphere quadrature (``sh``), the dG matrices M, D, h
assembled by quadrature (``dg``) and the time steppers (``steppers``).  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg / reference arm may import or call
anything here.  The CUDA library never links, imports or calls it, and the two share no code.
"""
