"""Crack-map surrogate: a BF16 U-Net run and trained by libcem's kernels
(include/cem_surrogate.h).  Only argument marshalling and buffer management
happen here; PyTorch supplies device memory and the stream.

Network (per level l with C_l channels): two 3x3 convolutions with ReLU,
2x2 max pooling down; up: nearest 2x upsampling of level l+1 concatenated
with the level-l skip, two 3x3 convolutions with ReLU; a 1x1 head to one
logit; class-weighted binary cross-entropy, optionally plus a weighted soft
Dice term per image; Adam.  Activations NHWC BF16;
the input's 3 channels are padded to 8.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Sequence

import numpy as np

from . import cem as _cem

_v = C.c_void_p
_i = C.c_int
_l = C.c_long
_f = C.c_float

# name -> (restype, argtypes); every entry point of include/cem_surrogate.h
SG_SIGNATURES = {
    "cem_sg_conv3x3": (_i, [_v, _i, _i, _i, _i, _i, _v, _v, _i, _i, _v, _i, _v, _i, _i, _v]),
    "cem_sg_wgrad_workspace": (_l, [_i, _i, _i, _i, _i]),
    "cem_sg_conv3x3_wgrad": (_i, [_v, _i, _v, _i, _i, _i, _i, _i, _i, _v, _v, _v, _l, _v]),
    "cem_sg_relu_bwd": (_i, [_v, _i, _v, _i, _l, _i, _v]),
    "cem_sg_maxpool2": (_i, [_v, _i, _i, _i, _i, _i, _v, _v]),
    "cem_sg_maxpool2_bwd": (_i, [_v, _i, _v, _v, _i, _i, _i, _i, _i, _i, _i, _v, _v]),
    "cem_sg_upsample2": (_i, [_v, _i, _i, _i, _i, _v, _i, _i, _v]),
    "cem_sg_upsample2_bwd": (_i, [_v, _i, _i, _i, _i, _i, _v, _i, _v, _v]),
    "cem_sg_head_fwd": (_i, [_v, _i, _i, _v, _v, _v, _v]),
    "cem_sg_head_workspace": (_l, [_i, _i]),
    "cem_sg_head_bwd": (_i, [_v, _i, _i, _v, _v, _v, _v, _v, _v, _l, _v]),
    "cem_sg_bce_workspace": (_l, [_l]),
    "cem_sg_bce": (_i, [_v, _v, _l, _f, _v, _v, _v, _l, _v]),
    "cem_sg_dice_workspace": (_l, [_i, _l]),
    "cem_sg_dice": (_i, [_v, _v, _i, _l, _f, _f, _v, _v, _v, _l, _v]),
    "cem_sg_adam": (_i, [_v, _v, _v, _v, _l, _f, _f, _f, _f, _i, _v, _v, _i, _i, _v]),
    "cem_sg_to_bf16": (_i, [_v, _l, _v, _v]),
    "cem_sg_set_gemm_path": (_i, [_i]),
    "cem_sg_timeouts": (_i, [C.POINTER(_i)]),
}

_SG = None


def sg():
    """libcem.so with the surrogate signatures set; raises if not built."""
    global _SG
    if _SG is None:
        L = _cem.lib()
        for name, (res, args) in SG_SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _SG = L
    return _SG


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with {rc}")


def timeouts() -> int:
    """Tensor-core CTAs whose bounded MMA wait gave up since the library was
    loaded (their outputs are invalid).  Synchronises with the device."""
    n = C.c_int(0)
    _ok(sg().cem_sg_timeouts(C.byref(n)), "cem_sg_timeouts")
    return n.value


def check_timeouts(before: int, what: str) -> int:
    """Raises if the time-out count grew past `before` during `what`; returns
    the current count."""
    now = timeouts()
    if now != before:
        raise RuntimeError(f"{now - before} tensor-core wait(s) gave up during {what}: "
                           "its results are invalid")
    return now


def _p(t, off_elems=0):
    """Device address of tensor t, plus an element offset."""
    return t.data_ptr() + off_elems * t.element_size()


class UNet:
    """U-Net with its buffers for one batch shape (B, H, W)."""

    def __init__(self, B: int, H: int, W: int, chans: Sequence[int] = (32, 64, 128, 256),
                 seed: int = 0, device: int = 0, pos_weight: float = 1.0, lr: float = 1e-3,
                 dice: float = 0.0, dice_eps: float = 1.0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.chans = list(chans)
        L = self.L = len(chans)
        if H % (1 << (L - 1)) or W % (1 << (L - 1)):
            raise ValueError("H and W must be divisible by 2^(levels-1)")
        if any(c % 8 for c in chans) or chans[0] > 32:
            raise ValueError("channels must be multiples of 8, level 0 at most 32")
        self.B, self.H, self.W = B, H, W
        self.pos_weight = float(pos_weight)
        self.dice, self.dice_eps = float(dice), float(dice_eps)
        self.lr = lr
        self.step_count = 0
        self.cin = 8
        rng = np.random.default_rng(seed)
        self.convs = {}
        order = []
        c = self.cin
        for l, ch in enumerate(chans):
            order += [(f"e{l}a", c, ch), (f"e{l}b", ch, ch)]
            c = ch
        for l in range(L - 2, -1, -1):
            order += [(f"d{l}a", c + chans[l], chans[l]), (f"d{l}b", chans[l], chans[l])]
            c = chans[l]
        f32, bf = torch.float32, torch.bfloat16
        for name, cin, cout in order:
            fan_in = 9 * (3 if name == "e0a" else cin)
            w = rng.standard_normal((cout, 3, 3, cin)) * math.sqrt(2.0 / fan_in)
            if name == "e0a":
                w[..., 3:] = 0.0  # padded input channels
            p = {"cin": cin, "cout": cout,
                 "w": torch.tensor(w, dtype=f32, device=self.dev),
                 "b": torch.zeros(cout, dtype=f32, device=self.dev)}
            for k in ("gw", "mw", "vw"):
                p[k] = torch.zeros_like(p["w"])
            for k in ("gb", "mb", "vb"):
                p[k] = torch.zeros_like(p["b"])
            p["wb"] = torch.empty((cout, 3, 3, cin), dtype=bf, device=self.dev)
            p["wt"] = torch.empty((cin, 3, 3, cout), dtype=bf, device=self.dev)
            self.convs[name] = p
        c0 = chans[0]
        hw = rng.standard_normal(c0) * math.sqrt(2.0 / c0) * 0.1
        self.head = {"w": torch.tensor(hw, dtype=f32, device=self.dev),
                     "b": torch.zeros(1, dtype=f32, device=self.dev)}
        for k in ("gw", "mw", "vw"):
            self.head[k] = torch.zeros_like(self.head["w"])
        for k in ("gb", "mb", "vb"):
            self.head[k] = torch.zeros_like(self.head["b"])
        self._refresh_copies()
        self._alloc()

    # -------------------------------------------------------------- buffers
    def _alloc(self):
        torch = self.torch
        bf = torch.bfloat16
        B, L, ch = self.B, self.L, self.chans
        self.dims = [(self.H >> l, self.W >> l) for l in range(L)]
        self.P = [B * h * w for h, w in self.dims]
        e = lambda n, c: torch.empty((n, c), dtype=bf, device=self.dev)
        self.x8 = e(self.P[0], 8)
        self.ea = [e(self.P[l], ch[l]) for l in range(L)]
        self.ldcat = [ch[l + 1] + ch[l] for l in range(L - 1)]
        self.cat = [e(self.P[l], self.ldcat[l]) for l in range(L - 1)]
        self.eb_bot = e(self.P[L - 1], ch[L - 1])
        self.pool = [e(self.P[l + 1], ch[l]) for l in range(L - 1)]
        self.da = [e(self.P[l], ch[l]) for l in range(L - 1)]
        self.db = [e(self.P[l], ch[l]) for l in range(L - 1)]
        self.gA = [e(self.P[l], ch[l]) for l in range(L)]
        self.gB = [e(self.P[l], ch[l]) for l in range(L)]
        self.gcat = [e(self.P[l], self.ldcat[l]) for l in range(L - 1)]
        self.gpool = [e(self.P[l + 1], ch[l]) for l in range(L - 1)]
        self.z = torch.empty(self.P[0], dtype=torch.float32, device=self.dev)
        self.dz = torch.empty_like(self.z)
        self.loss = torch.zeros(2, dtype=torch.float32, device=self.dev)
        L_ = sg()
        need = [L_.cem_sg_head_workspace(self.P[0], ch[0]), L_.cem_sg_bce_workspace(self.P[0]),
                L_.cem_sg_dice_workspace(B, self.P[0] // B)]
        for name, p in self.convs.items():
            l = int(name[1])
            h, w = self.dims[l]
            need.append(L_.cem_sg_wgrad_workspace(B, h, w, p["cin"], p["cout"]))
        self.ws_bytes = int(max(need))
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.dev)

    def _stream(self):
        return self.torch.cuda.current_stream(self.dev).cuda_stream

    def _refresh_copies(self):
        """BF16 and transposed-flipped copies of the masters (Adam with lr 0
        and a zero gradient leaves the weights and moments unchanged)."""
        st = self._stream()
        L_ = sg()
        for p in self.convs.values():
            p["gw"].zero_()
            n = p["w"].numel()
            _ok(L_.cem_sg_adam(_p(p["w"]), _p(p["gw"]), _p(p["mw"]), _p(p["vw"]), n, 0.0, 0.9,
                               0.999, 1e-8, 1, _p(p["wb"]), _p(p["wt"]), p["cout"], p["cin"], st),
                "adam")

    # -------------------------------------------------------------- forward
    def set_input(self, x8):
        """x8: device tensor [B*H*W, 8] BF16 (or FP32, converted here)."""
        torch = self.torch
        if x8.dtype == torch.bfloat16:
            self.x8.copy_(x8.reshape(self.P[0], 8))
        else:
            src = x8.reshape(-1).to(torch.float32).contiguous()
            _ok(sg().cem_sg_to_bf16(_p(src), src.numel(), _p(self.x8), self._stream()), "to_bf16")

    def _conv(self, name, x, ldx, y, ldy, yoff, relu=1, H=None, W=None, Cin=None):
        p = self.convs[name]
        _ok(sg().cem_sg_conv3x3(_p(x), self.B, H, W, Cin if Cin else p["cin"], ldx, _p(p["wb"]),
                                _p(p["b"]), p["cout"], relu, None, 0, _p(y), ldy, yoff,
                                self._stream()), "conv " + name)

    def forward(self):
        """Logits self.z [B*H*W] (FP32) of the current input."""
        L_, st, ch, L = sg(), self._stream(), self.chans, self.L
        h_in, ld_in = self.x8, 8
        for l in range(L):
            H, W = self.dims[l]
            self._conv(f"e{l}a", h_in, ld_in, self.ea[l], ch[l], 0, H=H, W=W)
            if l < L - 1:
                self._conv(f"e{l}b", self.ea[l], ch[l], self.cat[l], self.ldcat[l], ch[l + 1],
                           H=H, W=W)
                h2, w2 = self.dims[l + 1]
                _ok(L_.cem_sg_maxpool2(_p(self.cat[l], ch[l + 1]), self.ldcat[l], self.B, h2, w2,
                                       ch[l], _p(self.pool[l]), st), "maxpool")
                h_in, ld_in = self.pool[l], ch[l]
            else:
                self._conv(f"e{l}b", self.ea[l], ch[l], self.eb_bot, ch[l], 0, H=H, W=W)
        h = self.eb_bot
        for l in range(L - 2, -1, -1):
            H, W = self.dims[l]
            h2, w2 = self.dims[l + 1]
            _ok(L_.cem_sg_upsample2(_p(h), self.B, h2, w2, ch[l + 1], _p(self.cat[l]),
                                    self.ldcat[l], 0, st), "upsample")
            self._conv(f"d{l}a", self.cat[l], self.ldcat[l], self.da[l], ch[l], 0, H=H, W=W)
            self._conv(f"d{l}b", self.da[l], ch[l], self.db[l], ch[l], 0, H=H, W=W)
            h = self.db[l]
        _ok(L_.cem_sg_head_fwd(_p(h), self.P[0], ch[0], _p(self.head["w"]), _p(self.head["b"]),
                               _p(self.z), st), "head")
        return self.z

    # ------------------------------------------------------------- backward
    def _wgrad(self, name, x, ldx, dy, lddy, H, W):
        p = self.convs[name]
        _ok(sg().cem_sg_conv3x3_wgrad(_p(x), ldx, _p(dy), lddy, self.B, H, W, p["cin"], p["cout"],
                                      _p(p["gw"]), _p(p["gb"]), _p(self.ws), self.ws_bytes,
                                      self._stream()), "wgrad " + name)

    def _dgrad(self, name, dy, out, H, W, mask=None):
        """out = data gradient of conv `name` (dense [P, cin]); zero where
        mask (the conv's input, a ReLU output) is <= 0 when given."""
        p = self.convs[name]
        _ok(sg().cem_sg_conv3x3(_p(dy), self.B, H, W, p["cout"], p["cout"], _p(p["wt"]), None,
                                p["cin"], 0, None if mask is None else _p(mask),
                                p["cin"], _p(out), p["cin"], 0, self._stream()),
            "dgrad " + name)

    def backward(self, dz=None):
        """Gradients of sum(dz * z) into every parameter's gw / gb; dz
        defaults to the loss gradient left by loss().  Every ReLU's gradient
        mask is applied by the kernel that produces the gradient (head, data
        gradients, upsampling and pooling gradients)."""
        L_, st, ch, L = sg(), self._stream(), self.chans, self.L
        dz = self.dz if dz is None else dz
        hd = self.head
        _ok(L_.cem_sg_head_bwd(_p(self.db[0] if L > 1 else self.eb_bot), self.P[0], ch[0],
                               _p(hd["w"]), _p(dz), _p(self.gA[0]), _p(hd["gw"]), _p(hd["gb"]),
                               _p(self.ws), self.ws_bytes, st), "head_bwd")
        for l in range(L - 1):
            H, W = self.dims[l]
            self._wgrad(f"d{l}b", self.da[l], ch[l], self.gA[l], ch[l], H, W)
            self._dgrad(f"d{l}b", self.gA[l], self.gB[l], H, W, mask=self.da[l])
            self._wgrad(f"d{l}a", self.cat[l], self.ldcat[l], self.gB[l], ch[l], H, W)
            self._dgrad(f"d{l}a", self.gB[l], self.gcat[l], H, W)
            h2, w2 = self.dims[l + 1]
            up_in = self.db[l + 1] if l + 1 < L - 1 else self.eb_bot
            _ok(L_.cem_sg_upsample2_bwd(_p(self.gcat[l]), self.ldcat[l], self.B, h2, w2, ch[l + 1],
                                        _p(up_in), ch[l + 1], _p(self.gA[l + 1]), st),
                "upsample_bwd")
        for l in range(L - 1, -1, -1):
            H, W = self.dims[l]
            if l < L - 1:
                h2, w2 = self.dims[l + 1]
                _ok(L_.cem_sg_maxpool2_bwd(_p(self.cat[l], ch[l + 1]), self.ldcat[l],
                                           _p(self.gpool[l]), _p(self.gcat[l], ch[l + 1]),
                                           self.ldcat[l], 0, self.B, h2, w2, ch[l], 1,
                                           _p(self.gA[l]), st), "maxpool_bwd")
            self._wgrad(f"e{l}b", self.ea[l], ch[l], self.gA[l], ch[l], H, W)
            self._dgrad(f"e{l}b", self.gA[l], self.gB[l], H, W, mask=self.ea[l])
            if l == 0:
                self._wgrad("e0a", self.x8, 8, self.gB[0], ch[0], H, W)
            else:
                self._wgrad(f"e{l}a", self.pool[l - 1], ch[l - 1], self.gB[l], ch[l], H, W)
                self._dgrad(f"e{l}a", self.gB[l], self.gpool[l - 1], H, W)

    # ----------------------------------------------------------------- loss
    def loss_and_grad(self, target_u8):
        """Weighted BCE of self.z against target (device uint8 [B*H*W]), plus
        dice * (1 - mean soft Dice of the B images) when dice > 0; leaves
        d loss / d z in self.dz.  Returns the loss tensor (device; [0] the
        BCE, [1] the Dice term, zero without it)."""
        _ok(sg().cem_sg_bce(_p(self.z), _p(target_u8), self.P[0], self.pos_weight, _p(self.dz),
                            _p(self.loss), _p(self.ws), self.ws_bytes, self._stream()), "bce")
        if self.dice > 0:
            _ok(sg().cem_sg_dice(_p(self.z), _p(target_u8), self.B, self.P[0] // self.B,
                                 self.dice, self.dice_eps, _p(self.dz), _p(self.loss, 1),
                                 _p(self.ws), self.ws_bytes, self._stream()), "dice")
        return self.loss

    def adam_step(self, lr=None, b1=0.9, b2=0.999, eps=1e-8):
        lr = self.lr if lr is None else lr
        self.step_count += 1
        t, st, L_ = self.step_count, self._stream(), sg()
        for p in self.convs.values():
            _ok(L_.cem_sg_adam(_p(p["w"]), _p(p["gw"]), _p(p["mw"]), _p(p["vw"]), p["w"].numel(),
                               lr, b1, b2, eps, t, _p(p["wb"]), _p(p["wt"]), p["cout"], p["cin"],
                               st), "adam")
            _ok(L_.cem_sg_adam(_p(p["b"]), _p(p["gb"]), _p(p["mb"]), _p(p["vb"]), p["b"].numel(),
                               lr, b1, b2, eps, t, None, None, 0, 0, st), "adam")
        h = self.head
        _ok(L_.cem_sg_adam(_p(h["w"]), _p(h["gw"]), _p(h["mw"]), _p(h["vw"]), h["w"].numel(), lr,
                           b1, b2, eps, t, None, None, 0, 0, st), "adam")
        _ok(L_.cem_sg_adam(_p(h["b"]), _p(h["gb"]), _p(h["mb"]), _p(h["vb"]), 1, lr, b1, b2, eps,
                           t, None, None, 0, 0, st), "adam")

    def train_step(self, target_u8):
        self.forward()
        loss = self.loss_and_grad(target_u8)
        self.backward()
        self.adam_step()
        return loss

    # --------------------------------------------------------------- params
    def params_numpy(self):
        """FP32 master parameters as numpy arrays, named like the oracle's
        (input channels beyond the first three dropped from e0a)."""
        out = {}
        for name, p in self.convs.items():
            w = p["w"].detach().cpu().numpy().astype(np.float64)
            if name == "e0a":
                w = w[..., :3]
            out[name + ".w"] = w
            out[name + ".b"] = p["b"].detach().cpu().numpy().astype(np.float64)
        out["out.w"] = self.head["w"].detach().cpu().numpy().astype(np.float64).reshape(1, 1, 1, -1)
        out["out.b"] = self.head["b"].detach().cpu().numpy().astype(np.float64)
        return out

    def grads_numpy(self):
        out = {}
        for name, p in self.convs.items():
            g = p["gw"].detach().cpu().numpy().astype(np.float64)
            if name == "e0a":
                g = g[..., :3]
            out[name + ".w"] = g
            out[name + ".b"] = p["gb"].detach().cpu().numpy().astype(np.float64)
        out["out.w"] = self.head["gw"].detach().cpu().numpy().astype(np.float64).reshape(1, 1, 1, -1)
        out["out.b"] = self.head["gb"].detach().cpu().numpy().astype(np.float64)
        return out
