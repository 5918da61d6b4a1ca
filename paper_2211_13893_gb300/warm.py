"""Learned warm start of the local eigensolver (include/msgfem_warm.h).

Driver code only: it moves device buffers between the calls of the library
(features and aligned eigenvector targets from an MS-GFEM handle, training and
inference of one network per subdomain position, start blocks back into the
handle).  All arithmetic runs in the library's kernels.

Per subdomain position p (subdomain p of every instance of a batched handle)
one network maps the ply-angle perturbation on the elements of Omega*_p
(scaled by 1 / sd) to the wanted non-rigid eigenvectors restricted to the
interface rows B2, as a [n2][8] block (columns beyond the wanted count are
zero).  Targets are rotated onto the nominal (unperturbed) eigenvectors by
orthogonal Procrustes, which removes their sign and rotation freedom; the
output bias starts at that nominal block, so an untrained network reproduces
nominal-basis reuse.  Inference for a batched handle runs one forward pass
per position over all instances.
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
        self.S = getattr(m, "instances", 1)
        self.P = m.N // self.S                                          # positions
        self.sizes = [m.warm_sizes(p, n_loc) for p in range(self.P)]   # (n2, nw) per position
        self.dev = torch.device("cuda")
        self.stream = stream
        self.nfeat = None
        self.nominal = []
        self.nets = []
        self.hidden = tuple(hidden)
        self.seed = seed
        self.max_batch = max(max_batch, self.S)

    def size(self, j):
        return self.sizes[j % self.P]

    # ---- data from the handle -------------------------------------------------
    def features(self, dtheta):
        """Device float32 [N][nfeat] features of the perturbation fields dtheta
        (device float64, one field per instance)."""
        torch = self.torch
        if self.nfeat is None:
            self.nfeat = self.m.warm_features(None, self.scale, None, 0)
        feat = torch.empty((self.m.N, self.nfeat), dtype=torch.float32, device=self.dev)
        self.m.warm_features(dtheta, self.scale, feat, self.nfeat)
        return feat

    def targets(self, ref=True):
        """Per subdomain j: device float32 [n2][KB] eigenvector block of the last
        local stage (Procrustes-aligned to the nominal block of its position)."""
        torch = self.torch
        out = []
        for j in range(self.m.N):
            n2, _ = self.size(j)
            t = torch.empty((n2, KB), dtype=torch.float32, device=self.dev)
            self.m.warm_targets(j, t, KB, self.nominal[j % self.P] if (ref and self.nominal) else None)
            out.append(t)
        return out

    def set_nominal(self):
        """Record the last local stage's eigenvectors of instance 0 as the nominal blocks."""
        t = self.targets(ref=False)
        self.nominal = [t[p].clone() for p in range(self.P)]

    # ---- the networks ---------------------------------------------------------
    def _init_params(self, p):
        n2, _ = self.sizes[p]
        sizes = [self.nfeat, *self.hidden, n2 * KB]
        rng = np.random.default_rng(self.seed + 7919 * p)
        parts = []
        for l in range(len(sizes) - 1):
            fan_in, fan_out = sizes[l], sizes[l + 1]
            last = l + 2 == len(sizes)
            w = rng.standard_normal((fan_out, fan_in)) / np.sqrt(fan_in) * (0.01 if last else 1.0)
            b = self.nominal[p].reshape(-1).cpu().numpy() if last else np.zeros(fan_out)
            parts += [w.ravel(), b]
        return sizes, np.concatenate(parts).astype(np.float32)

    def build(self):
        if self.nfeat is None:
            self.nfeat = self.m.warm_features(None, self.scale, None, 0)
        self.nets = []
        for p in range(self.P):
            sizes, w = self._init_params(p)
            self.nets.append(Net(sizes, self.max_batch, w, self.stream))

    def fit(self, X, T, steps=4000, lr=3e-4, batch=64, seed=0):
        """X: device [samples][P][nfeat]; T: list over positions of device
        [samples][n2 * KB].  Returns the final minibatch losses."""
        torch = self.torch
        if not self.nets:
            self.build()
        n = X.shape[0]
        g = torch.Generator(device="cpu")
        g.manual_seed(seed)
        losses = []
        Xp = [X[:, p, :].contiguous() for p in range(self.P)]
        for step in range(steps):
            idx = torch.randperm(n, generator=g)[:min(batch, n)].to(self.dev)
            last = step + 1 == steps
            for p, net in enumerate(self.nets):
                xb = Xp[p].index_select(0, idx).contiguous()
                tb = T[p].index_select(0, idx).contiguous()
                lo = net.adam_step(xb, tb, xb.shape[0], lr, want_loss=last)
                if last:
                    losses.append(lo)
        return losses

    def predict(self, feat):
        """Start blocks (device float32 [n2][KB]) for every subdomain of the
        handle from its features [N][nfeat]: one forward pass per position."""
        torch = self.torch
        out = [None] * self.m.N
        fv = feat.view(self.S, self.P, -1)
        for p, net in enumerate(self.nets):
            n2, _ = self.sizes[p]
            y = torch.empty((self.S, n2 * KB), dtype=torch.float32, device=self.dev)
            net.forward(fv[:, p, :].contiguous(), y, self.S)
            for i in range(self.S):
                out[i * self.P + p] = y[i].view(n2, KB)
        return out

    def nominal_blocks(self):
        """The nominal blocks for every subdomain of the handle (nominal-basis reuse)."""
        return [self.nominal[j % self.P] for j in range(self.m.N)]

    def apply(self, blocks):
        """Register start blocks (or None for the cold start) with the handle."""
        for j in range(self.m.N):
            _, nw = self.size(j)
            if blocks is None or blocks[j] is None:
                self.m.set_start_block(j, None)
            else:
                self.m.set_start_block(j, blocks[j], KB, min(nw, KB))
