"""Low-rank far field of A(k), oracle side: the H-matrix route the paper takes for its largest
problems (Section 4, Example 3: the matrices are stored as H-matrices, compressed by adaptive
cross approximation). TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline).

The paper names the technique but not its parameters; the readings here are the textbook
ones, written out plainly:

* Cluster tree: the panels (by centroid) are split recursively at the middle of their
  order along the longest axis of their centroids' bounding box (ties by index) until a
  cluster holds at most ``leaf`` panels.
* Geometry of a cluster: the axis-aligned box of all vertices of its panels; diam = the box
  diagonal, dist = the distance between two boxes.
* Block partition, from (root, root): a pair is admissible (far) when
  max(diam(tau), diam(sigma)) <= eta dist(tau, sigma) (and, when a leaf size is given,
  both clusters hold more than two leaves of panels: smaller admissible blocks are cheaper
  dense); a pair of leaves that is not admissible is dense (near); otherwise the pair is
  split into the pairs of children (a leaf stays as it is). The blocks cover every (i, l)
  exactly once.
* Adaptive cross approximation with partial pivoting on a far block, entries A_il(k) of
  the 7-point rule: from row i* (first row of tau), residual row
  r = A[i*, sigma] - sum_p u_p[i*] w_p, pivot column j* = argmax |r|, w_k = r / r[j*],
  u_k = A[tau, j*] - sum_p u_p w_p[j*]; the squared Frobenius norm of the approximation is
  updated exactly, and the iteration stops when ||u_k|| ||w_k|| <= eps ||S_k||_F (or at
  rank rmax, or when every row has been used); the next row is argmax |u_k| over the unused
  rows. Block ~ U W^T (no conjugation).
"""
import numpy as np

from . import assembly


def _boxes(mesh, idx):
    v = mesh.xyz[mesh.tri[idx]].reshape(-1, 3)
    return v.min(0), v.max(0)


def cluster_tree(mesh, leaf=32):
    """Clusters as (index array, children, lo, hi) in a list; the root is cluster 0."""
    c = mesh.xyz[mesh.tri].mean(axis=1)
    clusters = []

    def build(idx):
        me = len(clusters)
        lo, hi = _boxes(mesh, idx)
        clusters.append([idx, [], lo, hi])
        if idx.size > leaf:
            cl, ch = c[idx].min(0), c[idx].max(0)
            axis = int(np.argmax(ch - cl))
            order = np.lexsort((idx, c[idx, axis]))
            sidx = idx[order]
            half = sidx.size // 2
            a = build(sidx[:half])
            b = build(sidx[half:])
            clusters[me][1] = [a, b]
        return me

    build(np.arange(mesh.n))
    return clusters


def _diam(cl):
    return float(np.linalg.norm(cl[3] - cl[2]))


def _dist(a, b):
    gap = np.maximum(0.0, np.maximum(a[2] - b[3], b[2] - a[3]))
    return float(np.linalg.norm(gap))


def blocks(clusters, eta=1.0, leaf=None):
    """Block list: (tau, sigma, far) cluster numbers. With ``leaf``, an admissible pair is
    far only when both clusters hold more than 2 leaf panels (smaller ones stay dense)."""
    out = []

    def split(t, s):
        A, B = clusters[t], clusters[s]
        big = leaf is None or min(A[0].size, B[0].size) > 2 * leaf
        if max(_diam(A), _diam(B)) <= eta * _dist(A, B) and big:
            out.append((t, s, True))
            return
        if not A[1] and not B[1]:
            out.append((t, s, False))
            return
        ts = A[1] if A[1] else [t]
        ss = B[1] if B[1] else [s]
        for a in ts:
            for b in ss:
                split(a, b)

    split(0, 0)
    return out


def aca(entry_rows, entry_cols, m, n, eps, rmax, history=False):
    """ACA with partial pivoting. entry_rows(i) -> row i (n values), entry_cols(j) -> column j
    (m values), local indices. Returns U (m x r), W (n x r); with history, also the updated
    squared norms ||S_k||_F^2 after each step."""
    U = np.zeros((m, 0), complex)
    W = np.zeros((n, 0), complex)
    used = np.zeros(m, bool)
    i = 0
    norm2 = 0.0
    hist = []
    while U.shape[1] < min(rmax, m, n):
        used[i] = True
        r = entry_rows(i) - U[i, :] @ W.T
        j = int(np.argmax(np.abs(r)))
        if abs(r[j]) == 0.0:
            if used.all():
                break
            i = int(np.argmin(used))   # the first unused row
            continue
        w = r / r[j]
        u = entry_cols(j) - U @ W[j, :]
        # ||S_k||^2 = ||S_{k-1}||^2 + 2 Re sum_p (u_p^H u)(w_p^H w) + ||u||^2 ||w||^2
        cross = 2.0 * np.real(np.sum((U.conj().T @ u) * (W.conj().T @ w)))
        nu, nw = np.linalg.norm(u), np.linalg.norm(w)
        norm2 += cross + (nu * nw) ** 2
        hist.append(norm2)
        U = np.hstack([U, u[:, None]])
        W = np.hstack([W, w[:, None]])
        if nu * nw <= eps * np.sqrt(max(norm2, 0.0)):
            break
        cand = np.abs(u).copy()
        cand[used] = -1.0
        if cand.max() < 0.0:
            break
        i = int(np.argmax(cand))
    return (U, W, hist) if history else (U, W)


def compress(mesh, k, clusters, blist, eps=1e-6, rmax=64, op=None):
    """Per far block (U, W); per near block the dense block."""
    out = []
    for t, s, far in blist:
        rows, cols = clusters[t][0], clusters[s][0]
        if far:
            er = lambda i: assembly.entries(mesh, k, np.full(cols.size, rows[i]), cols, op=op)
            ec = lambda j: assembly.entries(mesh, k, rows, np.full(rows.size, cols[j]), op=op)
            out.append(aca(er, ec, rows.size, cols.size, eps, rmax))
        else:
            rr, cc = np.meshgrid(rows, cols, indexing="ij")
            out.append(assembly.entries(mesh, k, rr.ravel(), cc.ravel(), op=op).reshape(rows.size, cols.size))
    return out


def apply(clusters, blist, comp, V):
    """Y = A_H V."""
    Y = np.zeros((V.shape[0], V.shape[1]), complex)
    for (t, s, far), c in zip(blist, comp):
        rows, cols = clusters[t][0], clusters[s][0]
        if far:
            U, W = c
            Y[rows] += U @ (W.T @ V[cols])
        else:
            Y[rows] += c @ V[cols]
    return Y


def dense(clusters, blist, comp, n):
    """A_H as a dense matrix (small n only)."""
    A = np.zeros((n, n), complex)
    for (t, s, far), c in zip(blist, comp):
        rows, cols = clusters[t][0], clusters[s][0]
        A[np.ix_(rows, cols)] = c[0] @ c[1].T if far else c
    return A
