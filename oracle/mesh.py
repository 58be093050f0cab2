"""Mesh connectivity and affine geometry of the oracle (test infrastructure only).

Conventions (Sec. 2, "Preliminaries": affine simplices, facets shared by at
most two elements):

* each element's vertices are sorted by global id; x = X_0 + J xi with
  J[:, i] = X_{i+1} - X_0 (det J keeps its sign);
* local facet f is the facet opposite local vertex f;
* global facets are numbered by sorting their (sorted) global vertex tuples
  lexicographically;
* the owner of a facet is the element with the lower index; its outward
  normal is the global facet normal n_F.  orient[e, f] = +1 for the owner
  (and for boundary facets), -1 for the other element.
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, verts, elems):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.elems = np.sort(np.asarray(elems, dtype=np.int64), axis=1)
        self.dim = self.verts.shape[1]
        self.n_elem = self.elems.shape[0]
        d = self.dim
        E = self.n_elem
        # --- facets by brute-force matching of sorted vertex tuples --------
        table = {}
        for e in range(E):
            for f in range(d + 1):
                key = tuple(int(v) for v in np.delete(self.elems[e], f))
                table.setdefault(key, []).append((e, f))
        keys = sorted(table)
        self.n_facets = len(keys)
        self.facet_verts = np.array(keys, dtype=np.int64)
        self.facet_id = np.empty((E, d + 1), dtype=np.int64)
        self.nbr = -np.ones((E, d + 1), dtype=np.int64)
        self.nbr_facet = -np.ones((E, d + 1), dtype=np.int64)
        self.orient = np.ones((E, d + 1), dtype=np.int64)
        self.facet_owner = np.empty((self.n_facets, 2), dtype=np.int64)   # (element, local facet)
        for g, key in enumerate(keys):
            sides = sorted(table[key])
            if len(sides) > 2:
                raise ValueError("non-manifold facet")
            self.facet_owner[g] = sides[0]
            for (e, f) in sides:
                self.facet_id[e, f] = g
            if len(sides) == 2:
                (e0, f0), (e1, f1) = sides
                self.nbr[e0, f0], self.nbr_facet[e0, f0] = e1, f1
                self.nbr[e1, f1], self.nbr_facet[e1, f1] = e0, f0
                self.orient[e1, f1] = -1
        # --- affine geometry ---------------------------------------------------
        X = self.verts[self.elems]                      # [E, d+1, d]
        self.X = X
        self.J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))   # J[e][:, i] = X_{i+1} - X_0
        self.detJ = np.linalg.det(self.J)
        self.Jinv = np.linalg.inv(self.J)
        # outward unit normals and measures of the local facets
        self.normal = np.empty((E, d + 1, d))
        self.area = np.empty((E, d + 1))
        for f in range(d + 1):
            fv = [v for v in range(d + 1) if v != f]
            P0 = X[:, fv[0], :]
            if d == 2:
                t = X[:, fv[1], :] - P0
                nvec = np.stack([t[:, 1], -t[:, 0]], axis=1)
            else:
                nvec = np.cross(X[:, fv[1], :] - P0, X[:, fv[2], :] - P0)
            length = np.linalg.norm(nvec, axis=1)
            self.area[:, f] = length if d == 2 else 0.5 * length
            nvec = nvec / length[:, None]
            away = np.einsum("ed,ed->e", nvec, P0 - X[:, f, :])
            self.normal[:, f, :] = nvec * np.sign(away)[:, None]

    def to_physical(self, e, xi):
        """x = X_0 + J xi for element indices e [M] and reference points xi [M, d]."""
        return self.X[e, 0, :] + np.einsum("mab,mb->ma", self.J[e], xi)

    def to_reference(self, e, x):
        """Brute-force affine inversion xi = J^{-1} (x - X_0)."""
        return np.einsum("mab,mb->ma", self.Jinv[e], x - self.X[e, 0, :])

    def shortest_edge(self):
        X = self.X
        d = self.dim
        h = np.full(self.n_elem, np.inf)
        for a in range(d + 1):
            for b in range(a + 1, d + 1):
                h = np.minimum(h, np.linalg.norm(X[:, a] - X[:, b], axis=1))
        return h
