"""Learned coefficients: the coefficient network as a fast stand-in for the OIS fit.

Pipeline (every numerical step runs in the library's kernels; this module moves tensors):

1. Training pairs come from the plain method: reference stamps R (cut around stars of a
   rendered field, with an h-pixel margin), local coefficients a drawn per stamp, and
   I = R (x) K(a) + noise computed by svk_difference_batch (each stamp a frame of degree
   0), cropped to 64 x 64.
2. The network (svk_cnn_*) is trained with its own gradient and Adam kernels to map the
   normalised pair to a (standardised by the draw's mean and spread).
3. On a frame: stamps at star positions -> local predictions -> svk_cnn_field_fit (FP64
   polynomial field c[k][t]) -> svk_difference.  If the residual chi^2 per stamp pixel
   exceeds `fallback_ratio` times the noise floor, the FP64 fit (svk_fit_coeffs) replaces
   the prediction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import (SVK_BASIS_GAUSS, SVK_METHOD_BASIS, SVK_PREC_BF16X3, svk_build_basis, svk_cnn_adam_device_step,
               svk_cnn_field_fit, svk_cnn_forward, svk_cnn_gradient, svk_cnn_param_count, svk_cnn_workspace_size,
               svk_difference, svk_difference_batch, svk_fit_coeffs)

STAMP = 64
SKY = 1000.0
SCALE = 3000.0  # input normalisation: (counts - sky) / SCALE


@dataclass
class CoeffPrior:
    """Distribution of the local coefficients the network is trained on."""
    n_out: int
    mean0: float = 1.0
    sd0: float = 0.03
    sd: float = 0.02

    def mean(self, device):
        m = torch.zeros(self.n_out, device=device)
        m[0] = self.mean0
        return m

    def std(self, device):
        s = torch.full((self.n_out,), self.sd, device=device)
        s[0] = self.sd0
        return s


def normalise(R, I):
    """[n][64][64] counts -> network input [n][2][64][64]."""
    return torch.stack([(R - SKY) / SCALE, (I - SKY) / SCALE], dim=1).contiguous()


def cut_stamps(img, cx, cy, size):
    """size x size stamps of img (zero outside) centred on integer (cx, cy) (torch tensors)."""
    H, W = img.shape
    half = size // 2
    off = torch.arange(size, device=img.device) - half
    ys = cy[:, None] + off[None, :]
    xs = cx[:, None] + off[None, :]
    ok = (ys[:, :, None] >= 0) & (ys[:, :, None] < H) & (xs[:, None, :] >= 0) & (xs[:, None, :] < W)
    v = img[ys.clamp(0, H - 1)[:, :, None], xs.clamp(0, W - 1)[:, None, :]]
    return torch.where(ok, v, torch.zeros_like(v)).contiguous()


def make_pairs(R_field, cx, cy, a, basis, noise_sigma, gen, chunk=64):
    """(x [n][2][64][64], R stamps, I stamps): I = R (x) K(a) + noise by the basis form."""
    L = basis.shape[1]
    h = L // 2
    big = cut_stamps(R_field, cx, cy, STAMP + 2 * h)
    n = big.shape[0]
    Ibig = torch.empty_like(big)
    for s in range(0, n, chunk):
        items = [dict(R=big[i], I=None, D=Ibig[i], basis=basis, coeffs=a[i:i + 1].T.contiguous(), degree=0)
                 for i in range(s, min(n, s + chunk))]
        svk_difference_batch(items, precision=SVK_PREC_BF16X3)
    Rs = big[:, h:h + STAMP, h:h + STAMP]
    Is = Ibig[:, h:h + STAMP, h:h + STAMP] + noise_sigma * torch.randn(Rs.shape, device=Rs.device, generator=gen)
    return normalise(Rs, Is), Rs.contiguous(), Is.contiguous()


class CoefficientNetwork:
    def __init__(self, params: torch.Tensor, prior: CoeffPrior, batch: int = 256):
        self.params = params.contiguous()
        self.prior = prior
        self.n_out = prior.n_out
        assert params.numel() == svk_cnn_param_count(self.n_out)
        self.batch = batch
        self.ws = torch.empty(svk_cnn_workspace_size(batch, self.n_out), dtype=torch.uint8, device=params.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._bufs = None   # fixed batch, gradient and loss buffers of the training step
        self._graph = None  # the gradient call over those buffers, captured as a CUDA graph
        self._graph_key = None

    _HIST = 1 << 14  # steps whose losses the captured step keeps on the device

    def _step_graph(self, x, z, lr):
        """One training step over fixed buffers as a CUDA graph: gather the batch named by
        the index buffer, svk_cnn_gradient, store the loss at the step's slot of a device
        history ring, advance the device step count, Adam (svk_cnn_adam_device_step).
        Captured once per (inputs, learning rate); the kernels and their arguments are those
        of the eager step."""
        dev = x.device
        shape = (self.batch,) + tuple(x.shape[1:])
        if self._bufs is None or self._bufs["x"].shape != shape or self._bufs["x"].device != dev:
            self._bufs = {"idx": torch.zeros(self.batch, dtype=torch.int64, device=dev),
                          "x": torch.zeros(shape, dtype=torch.float32, device=dev),
                          "z": torch.zeros((self.batch, self.n_out), dtype=torch.float32, device=dev),
                          "grad": torch.zeros_like(self.params), "loss": torch.zeros(1, dtype=torch.float32, device=dev),
                          "step": torch.zeros(1, dtype=torch.int32, device=dev),
                          "hist": torch.zeros(self._HIST, dtype=torch.float32, device=dev)}
            self._graph_key = None
        b = self._bufs
        key = (x.data_ptr(), z.data_ptr(), tuple(x.shape), float(lr), self.params.data_ptr(), self.ws.data_ptr())
        if self._graph_key != key:
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):  # first library call outside the capture (lazy setup)
                svk_cnn_gradient(self.params, b["x"], b["z"], grad=b["grad"], loss=b["loss"], workspace=self.ws)
            torch.cuda.current_stream().wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                torch.index_select(x, 0, b["idx"], out=b["x"])
                torch.index_select(z, 0, b["idx"], out=b["z"])
                svk_cnn_gradient(self.params, b["x"], b["z"], grad=b["grad"], loss=b["loss"], workspace=self.ws)
                b["hist"].index_copy_(0, torch.remainder(b["step"], self._HIST).long(), b["loss"])
                b["step"].add_(1)
                svk_cnn_adam_device_step(self.params, self.m, self.v, b["grad"], b["step"], lr=lr)
            self._graph, self._graph_key = graph, key
        return self._graph, b

    def train(self, x, a, steps: int, lr: float = 1e-3, gen=None):
        """Adam on standardised targets; returns the per-step losses (device tensor)."""
        dev = x.device
        z = ((a - self.prior.mean(dev)) / self.prior.std(dev)).contiguous()
        x = x.contiguous()
        losses = torch.empty(steps, device=dev)
        graph, b = self._step_graph(x, z, lr)
        b["step"].fill_(self.step)
        n = x.shape[0]
        done = 0
        while done < steps:  # chunks of at most one history ring
            c = min(self._HIST, steps - done)
            for _ in range(c):
                torch.randint(0, n, (self.batch,), generator=gen, out=b["idx"])
                graph.replay()
            first = (self.step + done) % self._HIST
            head = min(c, self._HIST - first)
            losses[done:done + head].copy_(b["hist"][first:first + head])
            if head < c:
                losses[done + head:done + c].copy_(b["hist"][:c - head])
            done += c
        self.step += steps
        return losses

    def state_dict(self):
        """Everything training depends on: weights, Adam moments and step (device tensors,
        cloned), the prior and the batch size.  Save it with torch.save; with the state of
        the generator that draws the batches, training resumes bit for bit."""
        return {"params": self.params.clone(), "m": self.m.clone(), "v": self.v.clone(), "step": self.step,
                "prior": (self.prior.n_out, self.prior.mean0, self.prior.sd0, self.prior.sd), "batch": self.batch}

    @classmethod
    def from_state_dict(cls, sd, device=None):
        params = sd["params"] if device is None else sd["params"].to(device)
        net = cls(params.clone(), CoeffPrior(*sd["prior"]), batch=sd["batch"])
        net.m.copy_(sd["m"])
        net.v.copy_(sd["v"])
        net.step = int(sd["step"])
        return net

    def predict(self, x):
        dev = x.device
        out = []
        for s in range(0, x.shape[0], self.batch):
            xb = x[s:s + self.batch].contiguous()
            ws = self.ws if xb.shape[0] == self.batch else None
            out.append(svk_cnn_forward(self.params, xb, self.n_out, workspace=ws))
        z = torch.cat(out)
        return self.prior.mean(dev) + self.prior.std(dev) * z


def apply_to_frame(net, R, I, stamp_xy, basis, degree, noise_sigma, fit_stamp=41, fallback_ratio=2.0,
                   reference_noise_sigma=None):
    """Coefficients for a frame from the network, with the FP64 fit as fallback.

    noise_sigma is the noise of I, reference_noise_sigma that of R when it is independent
    of I's (default: the same; 0 when I was made from the noisy R itself).  The noise floor
    of the residual D is noise_sigma^2 + reference_noise_sigma^2 sum K^2.
    Returns dict(coeffs [N][T] float32, source "network"|"fit", chi2_per_px, floor)."""
    cx = stamp_xy[:, 0].long()
    cy = stamp_xy[:, 1].long()
    x = normalise(cut_stamps(R, cx, cy, STAMP), cut_stamps(I, cx, cy, STAMP))
    local = net.predict(x).contiguous()
    H, W = R.shape
    c64, info = svk_cnn_field_fit(local, stamp_xy, W, H, degree)
    coeffs = c64.float().contiguous()
    D = svk_difference(R, I, basis, coeffs, degree, method=SVK_METHOD_BASIS, precision=SVK_PREC_BF16X3)
    half = fit_stamp // 2
    Ds = cut_stamps(D, cx, cy, fit_stamp)
    Ds = Ds - Ds.mean(dim=(1, 2), keepdim=True)  # the background is not part of the prediction
    chi2 = float((Ds.double() ** 2).mean())
    # noise floor of D = R (x) K - I, with K ~ the unit-sum first stamp
    rs = noise_sigma if reference_noise_sigma is None else reference_noise_sigma
    floor = noise_sigma ** 2 + rs ** 2 * float((basis[0].double() ** 2).sum())
    out = dict(coeffs=coeffs, source="network", chi2_per_px=chi2, floor=floor, info=int(info.item()))
    if int(info.item()) >= 0 or chi2 > fallback_ratio * floor:
        co, _, finfo = svk_fit_coeffs(R, I, stamp_xy, fit_stamp, basis, degree, bg_degree=0)
        T = (degree + 1) * (degree + 2) // 2
        out["coeffs"] = co[:basis.shape[0] * T].reshape(basis.shape[0], T).float().contiguous()
        out["source"] = "fit"
        out["fit_info"] = int(finfo.item())
    return out
