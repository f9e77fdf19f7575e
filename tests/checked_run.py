"""Runs the parity cases on the bounds-checked build of the library (a
separate shared object, loaded in a process of its own): every index read
from an index table is tested against its array, and any entry out of range
would fail the synchronising calls.  Exit status 0 when all cases pass."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from paper_2607_20704_gb300 import amr, build, inputs  # noqa: E402
from parity import compare_all  # noqa: E402


def main():
    amr.load(build.build(checked=True))
    cases = [inputs.random_mesh(3, 6, seed=51), inputs.random_mesh(4, 6, seed=52).shuffled(2),
             inputs.sod(4, 6), inputs.sedov(4, 6, radii={5: 0.15, 6: 0.08})]
    for prob in cases:
        for precision in (8, 4):
            g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision,
                         refine_grad_rho=0.1, refine_grad_p=0.1)
            o = oracle.Mesh(*prob.mesh_args(), **prob.params())
            for _ in range(2):
                g.regrid()
                o.regrid(grad_rho=0.1, grad_p=0.1)
                g.advance(1, sync=True)
                o.advance(1)
            if precision == 8:  # FP32 flags come from FP32 states: meshes may differ
                for l in o.levels():
                    assert np.array_equal(g.read(l)[0], o.read(l)[0]), (prob.name, l)
                compare_all(g, o, 1e-11)
            else:
                g.sync()
            g.close()
    # the fused shared-memory level steps, cube and planar (blocks, 27-neighbour
    # ring, reflux slots)
    for ns, precision, planar in ((1, 8, 0), (2, 8, 0), (2, 4, 0), (4, 4, 0), (1, 8, 1), (2, 8, 1), (4, 8, 1),
                                  (4, 4, 1)):
        prob = cases[0]
        g = amr.Mesh(*prob.mesh_args(), **prob.params(), precision=precision, nsubgrid=ns, planar=planar,
                      tile=128, schedule=1)
        g.advance(2, sync=True)
        if precision == 8:
            o = oracle.Mesh(*prob.mesh_args(), **prob.params())
            o.advance(2)
            compare_all(g, o, 1e-11)
        g.close()
    b = amr.Mesh.batch(cases[:3])
    b.advance(2, sync=True)
    b.close()
    # the deepest hierarchy a handle holds (levels 2..15, 14-bit coordinates)
    deep = inputs.sedov(2, 15, radii={l: 3 * 2.0 ** -l for l in range(3, 16)}, centre=(0.3, 0.7, 0.55))
    for precision in (8, 4):
        g = amr.Mesh(*deep.mesh_args(), **deep.params(), precision=precision, tile=128, schedule=0, nsubgrid=0)
        g.advance(1, sync=True)
        if precision == 8:
            o = oracle.Mesh(*deep.mesh_args(), **deep.params())
            o.advance(1)
            compare_all(g, o, 1e-11)
        g.close()
    print("checked build: all cases passed")


if __name__ == "__main__":
    main()
