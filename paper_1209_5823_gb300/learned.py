"""Learned coefficients: the coefficient network as a fast stand-in for the OIS fit.

Pipeline (every numerical step runs in the library's kernels; this module moves tensors):

1. Training pairs come from the plain method: reference stamps R (cut around stars of a
   rendered field, with an h-pixel margin), local coefficients a drawn per stamp, and
   I = R (x) K(a) + noise computed by svk_difference_batch (each stamp a frame of degree
   0), cropped to 64 x 64.
2. The network (svk_cnn_*) is trained with its own gradient and Adam kernels to map the
   normalised pair (svk_cut_stamps) to a (standardised by the draw's mean and spread,
   svk_cnn_standardise); a training step is one CUDA graph of library kernels that draws
   its batch on the device.
3. On a frame: stamps at star positions -> local predictions -> svk_cnn_field_fit (FP64
   polynomial field c[k][t]) -> svk_difference -> svk_stamp_residual.  If the residual
   chi^2 per stamp pixel exceeds `fallback_ratio` times the noise floor, the FP64 fit
   (svk_fit_coeffs) replaces the prediction.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import (SVK_METHOD_BASIS, SVK_PREC_BF16X3, svk_cnn_adam_device_step, svk_cnn_draw_batch, svk_cnn_field_fit,
               svk_cnn_forward, svk_cnn_gradient, svk_cnn_param_count, svk_cnn_standardise, svk_cnn_step_end,
               svk_cnn_workspace_size, svk_cut_stamps, svk_difference, svk_difference_batch, svk_fit_coeffs,
               svk_gather_rows, svk_stamp_residual)

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


def stamp_centres(cx, cy):
    """int32 [n][2] (x, y) centres from two integer tensors."""
    return torch.stack([cx, cy], dim=1).to(torch.int32).contiguous()


def network_input(R, I, xy, out=None):
    """The network's input [n][2][64][64]: stamps of R and I around the centres xy,
    (counts - sky) / SCALE, zero counts outside the frames (svk_cut_stamps)."""
    n = xy.shape[0]
    if out is None:
        out = torch.empty((n, 2, STAMP, STAMP), dtype=torch.float32, device=R.device)
    svk_cut_stamps(R, xy, STAMP, SKY, SCALE, out=out, stamp_stride=2 * STAMP * STAMP)
    svk_cut_stamps(I, xy, STAMP, SKY, SCALE, out=out[:, 1], stamp_stride=2 * STAMP * STAMP)
    return out


def cut_stamps(img, xy, size):
    """size x size stamps of img (zero outside) around the int32 [n][2] centres xy."""
    return svk_cut_stamps(img, xy, size)


def make_pairs(R_field, cx, cy, a, basis, noise_sigma, gen, chunk=64):
    """(x [n][2][64][64], R stamps, I stamps): I = R (x) K(a) + noise by the basis form.

    The reference stamps are cut with an h-pixel margin so that the convolution of their
    central 64 x 64 pixels sees the field around them; Gaussian noise of noise_sigma (the
    second epoch's own noise) is drawn from `gen`."""
    L = basis.shape[1]
    h = L // 2
    B = STAMP + 2 * h
    big = svk_cut_stamps(R_field, stamp_centres(cx, cy), B)
    n = big.shape[0]
    Ibig = torch.empty_like(big)
    for s in range(0, n, chunk):
        items = [dict(R=big[i], I=None, D=Ibig[i], basis=basis, coeffs=a[i:i + 1].T.contiguous(), degree=0)
                 for i in range(s, min(n, s + chunk))]
        svk_difference_batch(items, precision=SVK_PREC_BF16X3)
    Ibig += noise_sigma * torch.randn(Ibig.shape, device=Ibig.device, generator=gen)
    # the central 64 x 64 of every big stamp: the stack read as one image of n B rows
    ctr = torch.stack([torch.full((n,), B // 2, device=big.device, dtype=torch.int32),
                       torch.arange(n, device=big.device, dtype=torch.int32) * B + B // 2], dim=1)
    stackR, stackI = big.view(n * B, B), Ibig.view(n * B, B)
    x = network_input(stackR, stackI, ctr)
    return x, svk_cut_stamps(stackR, ctr, STAMP), svk_cut_stamps(stackI, ctr, STAMP)


class CoefficientNetwork:
    def __init__(self, params: torch.Tensor, prior: CoeffPrior, batch: int = 256, seed: int = 0):
        self.params = params.contiguous()
        self.prior = prior
        self.n_out = prior.n_out
        assert params.numel() == svk_cnn_param_count(self.n_out)
        self.batch = batch
        self.seed = int(seed)  # the batch draws of a run are fixed by (seed, step)
        self.ws = torch.empty(svk_cnn_workspace_size(batch, self.n_out), dtype=torch.uint8, device=params.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._bufs = None    # batch, gradient, loss, step and history buffers of the training step
        self._graphs = {}    # steps per replay -> captured CUDA graph
        self._graph_key = None

    _HIST = 1 << 14  # steps whose losses the captured step keeps on the device
    _GROUP = 8       # training steps captured in one graph

    def _step_graph(self, x, z, lr, k):
        """k training steps over fixed buffers as one CUDA graph, each step library kernels
        only: draw the batch on the device (svk_cnn_draw_batch, counter = the device step
        count), gather its inputs and targets (svk_gather_rows), svk_cnn_gradient, record
        the loss and advance the step count (svk_cnn_step_end), Adam with the device step
        count (svk_cnn_adam_device_step).  Captured once per (inputs, learning rate, k)."""
        dev = x.device
        shape = (self.batch,) + tuple(x.shape[1:])
        if self._bufs is None or self._bufs["x"].shape != shape or self._bufs["x"].device != dev:
            self._bufs = {"idx": torch.zeros(self.batch, dtype=torch.int64, device=dev),
                          "x": torch.zeros(shape, dtype=torch.float32, device=dev),
                          "z": torch.zeros((self.batch, self.n_out), dtype=torch.float32, device=dev),
                          "grad": torch.zeros_like(self.params), "loss": torch.zeros(1, dtype=torch.float32, device=dev),
                          "step": torch.zeros(1, dtype=torch.int32, device=dev),
                          "hist": torch.zeros(self._HIST, dtype=torch.float32, device=dev)}
            self._graphs, self._graph_key = {}, None
        b = self._bufs
        key = (x.data_ptr(), z.data_ptr(), tuple(x.shape), float(lr), self.params.data_ptr(), self.ws.data_ptr(),
               self.seed)
        if self._graph_key != key:
            self._graphs, self._graph_key = {}, key
        if k not in self._graphs:
            n = x.shape[0]
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):  # first library calls outside the capture (lazy setup)
                svk_cnn_gradient(self.params, b["x"], b["z"], grad=b["grad"], loss=b["loss"], workspace=self.ws)
                svk_cnn_draw_batch(self.seed, b["step"], n, b["idx"])
                svk_gather_rows(x, b["idx"], b["x"])
                scratch = torch.zeros(2, dtype=torch.int32, device=dev)
                svk_cnn_step_end(b["loss"], scratch[:1], b["hist"][:1].clone())
            torch.cuda.current_stream().wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                for _ in range(k):
                    svk_cnn_draw_batch(self.seed, b["step"], n, b["idx"])
                    svk_gather_rows(x, b["idx"], b["x"])
                    svk_gather_rows(z, b["idx"], b["z"])
                    svk_cnn_gradient(self.params, b["x"], b["z"], grad=b["grad"], loss=b["loss"], workspace=self.ws)
                    svk_cnn_step_end(b["loss"], b["step"], b["hist"])
                    svk_cnn_adam_device_step(self.params, self.m, self.v, b["grad"], b["step"], lr=lr)
            self._graphs[k] = graph
        return self._graphs[k], b

    def train(self, x, a, steps: int, lr: float = 1e-3):
        """Adam on standardised targets; returns the per-step losses (device tensor)."""
        dev = x.device
        z = svk_cnn_standardise(a, self.prior.mean(dev), self.prior.std(dev))
        x = x.contiguous()
        losses = torch.empty(steps, device=dev)
        g8, b = self._step_graph(x, z, lr, self._GROUP)
        g1, _ = self._step_graph(x, z, lr, 1)
        b["step"].fill_(self.step)
        done = 0
        while done < steps:  # chunks of at most one history ring
            c = min(self._HIST, steps - done)
            for _ in range(c // self._GROUP):
                g8.replay()
            for _ in range(c % self._GROUP):
                g1.replay()
            first = (self.step + done) % self._HIST
            head = min(c, self._HIST - first)
            losses[done:done + head].copy_(b["hist"][first:first + head])
            if head < c:
                losses[done + head:done + c].copy_(b["hist"][:c - head])
            done += c
        self.step += steps
        return losses

    def state_dict(self):
        """Everything training depends on: weights, Adam moments, step and the batch-draw
        seed (device tensors cloned), the prior and the batch size.  Save it with
        torch.save; training resumes bit for bit (the draws are fixed by seed and step)."""
        return {"params": self.params.clone(), "m": self.m.clone(), "v": self.v.clone(), "step": self.step,
                "seed": self.seed, "prior": (self.prior.n_out, self.prior.mean0, self.prior.sd0, self.prior.sd),
                "batch": self.batch}

    @classmethod
    def from_state_dict(cls, sd, device=None):
        params = sd["params"] if device is None else sd["params"].to(device)
        net = cls(params.clone(), CoeffPrior(*sd["prior"]), batch=sd["batch"], seed=sd.get("seed", 0))
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
        return svk_cnn_standardise(z, self.prior.mean(dev), self.prior.std(dev), inverse=True)


def apply_to_frame(net, R, I, stamp_xy, basis, degree, noise_sigma, fit_stamp=41, fallback_ratio=2.0,
                   reference_noise_sigma=None):
    """Coefficients for a frame from the network, with the FP64 fit as fallback.

    noise_sigma is the noise of I, reference_noise_sigma that of R when it is independent
    of I's (default: the same; 0 when I was made from the noisy R itself).  The noise floor
    of the residual D is noise_sigma^2 + reference_noise_sigma^2 sum K^2; the decision is
    svk_stamp_residual's (one device-to-host read).
    Returns dict(coeffs [N][T] float32, source "network"|"fit", chi2_per_px, floor)."""
    xy = stamp_xy.to(torch.int32).contiguous()
    local = net.predict(network_input(R, I, xy)).contiguous()
    H, W = R.shape
    c64, info = svk_cnn_field_fit(local, xy, W, H, degree)
    coeffs = c64.float().contiguous()
    D = svk_difference(R, I, basis, coeffs, degree, method=SVK_METHOD_BASIS, precision=SVK_PREC_BF16X3)
    rs = noise_sigma if reference_noise_sigma is None else reference_noise_sigma
    chk, fallback = svk_stamp_residual(D, xy, fit_stamp, basis[0], noise_sigma, rs, fallback_ratio, field_info=info)
    vals = torch.cat([chk, fallback.double(), info.double()]).cpu().tolist()
    out = dict(coeffs=coeffs, source="network", chi2_per_px=vals[0], floor=vals[1], info=int(vals[3]))
    if vals[2] != 0:
        co, _, finfo = svk_fit_coeffs(R, I, xy, fit_stamp, basis, degree, bg_degree=0)
        T = (degree + 1) * (degree + 2) // 2
        out["coeffs"] = co[:basis.shape[0] * T].reshape(basis.shape[0], T).float().contiguous()
        out["source"] = "fit"
        out["fit_info"] = int(finfo.item())
    return out
