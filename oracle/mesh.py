"""Structured laminated-beam mesh, boundary data and load vector.

Node (i, j, k) sits at (i hx, j hy, k t) and has global id
(i (NY+1) + j)(NZ+1) + k; its DoFs are 3 id + c (components blocked per node,
Sec. 2 "we block together displacements").  Element (i, j, k) spans nodes
i..i+1, j..j+1, k..k+1; layer k is ply k.

Boundary: Gamma_D is the x = 0 face (h = 0, all components clamped); the rest
of the boundary is Gamma_N; the x = L face carries a uniform traction g and
the other faces are traction-free (Eq. weak_form).
"""
import numpy as np

from .element import CORNERS


class BeamMesh:
    def __init__(self, NX, NY, NZ, hx, hy, t):
        self.NX, self.NY, self.NZ = NX, NY, NZ
        self.hx, self.hy, self.t = hx, hy, t
        self.n_nodes = (NX + 1) * (NY + 1) * (NZ + 1)
        self.n_dof = 3 * self.n_nodes

    @classmethod
    def from_config(cls, cfg):
        return cls(cfg.NX, cfg.NY, cfg.NZ, cfg.hx, cfg.hy, cfg.t)

    def node_id(self, i, j, k):
        return (np.asarray(i) * (self.NY + 1) + np.asarray(j)) * (self.NZ + 1) + np.asarray(k)

    def node_ijk(self, n):
        n = np.asarray(n)
        k = n % (self.NZ + 1)
        ij = n // (self.NZ + 1)
        return ij // (self.NY + 1), ij % (self.NY + 1), k

    def coords(self, n):
        i, j, k = self.node_ijk(n)
        return np.stack([i * self.hx, j * self.hy, k * self.t], axis=-1).astype(np.float64)

    def element_nodes(self, i, j, k):
        """Global node ids of element (i, j, k) in the ``CORNERS`` order (arrays broadcast)."""
        off = ((CORNERS + 1) // 2).astype(np.int64)
        i, j, k = (np.asarray(v)[..., None] for v in (i, j, k))
        return self.node_id(i + off[:, 0], j + off[:, 1], k + off[:, 2])

    def element_dofs(self, i, j, k):
        nodes = self.element_nodes(i, j, k)
        return (3 * nodes[..., :, None] + np.arange(3)).reshape(nodes.shape[:-1] + (24,))

    def dirichlet_dofs(self):
        """All DoFs of the clamped x = 0 face."""
        j, k = np.meshgrid(np.arange(self.NY + 1), np.arange(self.NZ + 1), indexing="ij")
        nodes = self.node_id(0, j.ravel(), k.ravel())
        return np.sort((3 * nodes[:, None] + np.arange(3)).ravel())

    def face_load(self, g):
        """b(v) = int_{x=L} g . v ds for a constant traction vector g.

        Each face quad of the x = L face is integrated with a 2x2 Gauss rule over
        the bilinear trace of the shape functions.
        """
        g = np.asarray(g, dtype=np.float64)
        b = np.zeros(self.n_dof)
        x, w = np.polynomial.legendre.leggauss(2)
        area_jac = self.hy * self.t / 4.0
        for j in range(self.NY):
            for k in range(self.NZ):
                nodes = [self.node_id(self.NX, j + dj, k + dk) for dj in (0, 1) for dk in (0, 1)]
                for a, (dj, dk) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
                    # bilinear face shape function of corner (dj, dk)
                    s = 0.0
                    for p in range(2):
                        for q in range(2):
                            Na = (1 + (2 * dj - 1) * x[p]) * (1 + (2 * dk - 1) * x[q]) / 4.0
                            s += Na * w[p] * w[q] * area_jac
                    b[3 * nodes[a]:3 * nodes[a] + 3] += s * g
        return b

    def compression_load(self, p):
        """Uniform compressive traction of magnitude p on x = L (g = (-p, 0, 0))."""
        return self.face_load((-p, 0.0, 0.0))



class HexMesh(BeamMesh):
    """Structured hexahedral mesh with arbitrary node coordinates.

    Same index space, numbering and boundary faces as ``BeamMesh`` (clamped
    i = 0 face, loaded i = NX face), but node (i, j, k) sits at
    ``xyz[i, j, k]`` and element (i, j, k) carries its own ply frame
    ``frames[i, j, k]`` (rows a0, a1, a2; see ``material.material_axes``).
    Used for the curved C-section spar.
    """

    general = True

    def __init__(self, xyz, frames):
        xyz = np.asarray(xyz, dtype=np.float64)
        NX, NY, NZ = (n - 1 for n in xyz.shape[:3])
        super().__init__(NX, NY, NZ, float("nan"), float("nan"), float("nan"))
        self.xyz = xyz
        self.frames = np.asarray(frames, dtype=np.float64)

    @classmethod
    def from_config(cls, cfg):
        from workloads.section import section_frames, section_nodes
        return cls(section_nodes(cfg), section_frames(cfg))

    def coords(self, n):
        i, j, k = self.node_ijk(n)
        return self.xyz[i, j, k]

    def element_corners(self, i, j, k):
        """8x3 corner coordinates of element (i, j, k) in the ``CORNERS`` order."""
        off = ((CORNERS + 1) // 2).astype(np.int64)
        return self.xyz[i + off[:, 0], j + off[:, 1], k + off[:, 2]]

    def face_load(self, g):
        """b(v) = int_{x=L} g . v ds over the i = NX face.

        Each face quad is the bilinear map X(s, r) = sum_a N_a(s, r) X_a of its
        four nodes; int N_a dA = int N_a |X_s x X_r| ds dr, taken with a 3x3
        Gauss rule (exact: the integrand is a polynomial of degree <= 2 in each
        variable on a planar quad).
        """
        g = np.asarray(g, dtype=np.float64)
        b = np.zeros(self.n_dof)
        x, w = np.polynomial.legendre.leggauss(3)
        corners = ((0, 0), (0, 1), (1, 0), (1, 1))
        for j in range(self.NY):
            for k in range(self.NZ):
                X = np.array([self.xyz[self.NX, j + dj, k + dk] for dj, dk in corners])
                nodes = [self.node_id(self.NX, j + dj, k + dk) for dj, dk in corners]
                sgn = np.array([(2 * dj - 1, 2 * dk - 1) for dj, dk in corners], dtype=np.float64)
                acc = np.zeros(4)
                for p in range(3):
                    for q in range(3):
                        s, r = x[p], x[q]
                        N = (1 + sgn[:, 0] * s) * (1 + sgn[:, 1] * r) / 4.0
                        dNs = sgn[:, 0] * (1 + sgn[:, 1] * r) / 4.0
                        dNr = (1 + sgn[:, 0] * s) * sgn[:, 1] / 4.0
                        Xs, Xr = dNs @ X, dNr @ X
                        acc += N * np.linalg.norm(np.cross(Xs, Xr)) * w[p] * w[q]
                for a in range(4):
                    b[3 * nodes[a]:3 * nodes[a] + 3] += acc[a] * g
        return b


def make_mesh(cfg):
    """The oracle mesh of a workload: a box beam or the curved C-section."""
    if getattr(cfg, "kind", "beam") == "section":
        return HexMesh.from_config(cfg)
    return BeamMesh.from_config(cfg)
