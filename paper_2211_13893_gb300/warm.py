"""Learned warm start of the local eigensolver (include/msgfem_warm.h).

Driver code only: it moves device buffers between the calls of the library
(features and aligned eigenvector targets from an MS-GFEM handle, training and
inference of one network per subdomain position, start blocks back into the
handle).  All arithmetic runs in the library's kernels.

Per subdomain j the network maps the ply-angle perturbation on the elements of
Omega*_j (scaled by 1 / sd) to the wanted non-rigid eigenvectors restricted to
the interface rows B2, as a [n2][8] block (columns beyond the wanted count are
zero).  Targets are rotated onto the nominal (unperturbed) eigenvectors by
orthogonal Procrustes, which removes their sign and rotation freedom; the
output bias starts at that nominal block, so an untrained network reproduces
nominal-basis reuse.
"""
import numpy as np

from .msgfem import Net

KB = 8   # width of the eigensolver's start block


class WarmStart:
    def __init__(self, m, n_loc, hidden=(32,), scale=1.0 / 3.0, seed=0, max_batch=512, stream=None):
        import torch
        self.torch = torch
        self.m = m
        self.n_loc = n_loc
        self.scale = float(scale)
        self.sizes = [m.warm_sizes(j, n_loc) for j in range(m.N)]   # (n2, nw)
        dev = torch.device("cuda")
        self.dev = dev
        self.stream = stream
        self.nfeat = None
        self.feat = None
        self.nominal = []
        self.nets = []
        self.hidden = tuple(hidden)
        self.seed = seed
        self.max_batch = max_batch

    # ---- data from the handle -------------------------------------------------
    def features(self, dtheta):
        """Device float32 [N][nfeat] features of the perturbation field dtheta (device float64)."""
        torch = self.torch
        if self.nfeat is None:
            self.nfeat = self.m.warm_features(None, self.scale, None, 0)
        feat = torch.empty((self.m.N, self.nfeat), dtype=torch.float32, device=self.dev)
        self.m.warm_features(dtheta, self.scale, feat, self.nfeat)
        return feat

    def targets(self, ref=True):
        """Per subdomain: device float32 [n2][KB] eigenvector blocks of the last local stage."""
        torch = self.torch
        out = []
        for j, (n2, _) in enumerate(self.sizes):
            t = torch.empty((n2, KB), dtype=torch.float32, device=self.dev)
            self.m.warm_targets(j, t, KB, self.nominal[j] if (ref and self.nominal) else None)
            out.append(t)
        return out

    def set_nominal(self):
        """Record the current local stage's eigenvectors as the nominal blocks."""
        self.nominal = [t.clone() for t in self.targets(ref=False)]

    # ---- the networks ---------------------------------------------------------
    def _init_params(self, j):
        n2, _ = self.sizes[j]
        sizes = [self.nfeat, *self.hidden, n2 * KB]
        rng = np.random.default_rng(self.seed + 7919 * j)
        parts = []
        for l in range(len(sizes) - 1):
            fan_in, fan_out = sizes[l], sizes[l + 1]
            last = l + 2 == len(sizes)
            w = rng.standard_normal((fan_out, fan_in)) / np.sqrt(fan_in) * (0.01 if last else 1.0)
            b = self.nominal[j].reshape(-1).cpu().numpy() if last else np.zeros(fan_out)
            parts += [w.ravel(), b]
        return sizes, np.concatenate(parts).astype(np.float32)

    def build(self):
        if self.nfeat is None:
            self.nfeat = self.m.warm_features(None, self.scale, None, 0)
        self.nets = []
        for j in range(self.m.N):
            sizes, p = self._init_params(j)
            self.nets.append(Net(sizes, self.max_batch, p, self.stream))

    def fit(self, X, T, steps=4000, lr=3e-4, batch=64, seed=0):
        """X: device [S][N][nfeat]; T: list over j of device [S][n2 * KB].  Returns final losses."""
        torch = self.torch
        if not self.nets:
            self.build()
        S = X.shape[0]
        g = torch.Generator(device="cpu")
        g.manual_seed(seed)
        losses = []
        Xj = [X[:, j, :].contiguous() for j in range(self.m.N)]
        for step in range(steps):
            idx = torch.randperm(S, generator=g)[:min(batch, S)].to(self.dev)
            last = step + 1 == steps
            for j, net in enumerate(self.nets):
                xb = Xj[j].index_select(0, idx).contiguous()
                tb = T[j].index_select(0, idx).contiguous()
                lo = net.adam_step(xb, tb, xb.shape[0], lr, want_loss=last)
                if last:
                    losses.append(lo)
        return losses

    def predict(self, feat):
        """Start blocks (device float32 [n2][KB] per subdomain) for one sample's features [N][nfeat]."""
        torch = self.torch
        out = []
        for j, net in enumerate(self.nets):
            n2, _ = self.sizes[j]
            y = torch.empty((1, n2 * KB), dtype=torch.float32, device=self.dev)
            net.forward(feat[j:j + 1].contiguous(), y, 1)
            out.append(y.view(n2, KB))
        return out

    def apply(self, blocks):
        """Register start blocks (or None for the cold start) with the handle."""
        for j, (n2, nw) in enumerate(self.sizes):
            if blocks is None or blocks[j] is None:
                self.m.set_start_block(j, None)
            else:
                self.m.set_start_block(j, blocks[j], KB, nw)
