"""Reader for the hand-written fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_sections(name):
    secs, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("["):
                cur = line[1:line.index("]")]
                secs[cur] = []
                continue
            secs[cur].append([float(x) for x in line.split()])
    return secs


def phi_small():
    s = read_sections("phi_small.txt")
    nt, na, nv, nf = (int(x) for x in s["dims"][0])

    def coo(rows):
        a = np.array(rows)
        return (a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), a[:, 2].astype(np.int32),
                a[:, 3].astype(np.float32))

    flat = lambda k: np.array([x for row in s[k] for x in row], np.float64)
    return dict(nt=nt, na=na, nv=nv, nf=nf, raw=coo(s["raw"]), voxel=coo(s["voxel"]), fiber=coo(s["fiber"]),
                atom=coo(s["atom"]), D=flat("D"), w=flat("w"), y=flat("y"), r=flat("r"), g=flat("g"))
