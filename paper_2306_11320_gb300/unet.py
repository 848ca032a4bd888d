"""The warm-start U-Net: a 4-level BF16 network trained and run by the library's own
tensor-core kernels (include/tpfnet.h).  This module only allocates buffers (torch
tensors), orders the kernel calls and marshals arguments; every layer, gradient and
optimizer update runs in CUDA.

Network (channels c0..c3, NHWC bf16, input channels padded to 32):
  e0 = relu(conv(relu(conv(x))))            e1 = ... (pool(e0))     e2 = ... (pool(e1))
  b  = relu(conv(relu(conv(pool(e2)))))
  d2 = relu(conv(relu(conv(cat(up(b), e2)))))   d1 = ... cat(up(d2), e1)   d0 = ... cat(up(d1), e0)
  out = head(d0)  (1x1, float32)
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .tpflbm import load_library

_vp, _ip, _ll, _fl = C.c_void_p, C.c_int, C.c_longlong, C.c_float
_fp, _dp = C.POINTER(C.c_float), C.POINTER(C.c_double)

SIGNATURES = {
    "tpfnet_conv3x3": [_vp, _ip, _ip, _ip, _ip, _vp, _vp, _ip, _ip, _vp, _vp],
    "tpfnet_conv3x3_tcgen05": [_ip, _ip, _ip, _ip, _ip],
    "tpfnet_conv3x3_wgrad_tcgen05": [_ip, _ip, _ip, _ip, _ip],
    "tpfnet_status": [],
    "tpfnet_conv3x3_dgrad": [_vp, _ip, _ip, _ip, _ip, _vp, _ip, _vp, _vp, _vp],
    "tpfnet_conv3x3_wgrad": [_vp, _vp, _ip, _ip, _ip, _ip, _ip, _vp, _vp, _vp],
    "tpfnet_relu_mask": [_vp, _vp, _ll, _vp],
    "tpfnet_pool": [_vp, _ip, _ip, _ip, _ip, _vp, _vp],
    "tpfnet_pool_back": [_vp, _ip, _ip, _ip, _ip, _vp, _ip, _vp],
    "tpfnet_up_into": [_vp, _ip, _ip, _ip, _ip, _vp, _ip, _ip, _vp],
    "tpfnet_up_back": [_vp, _ip, _ip, _ip, _ip, _ip, _ip, _vp, _vp],
    "tpfnet_channels": [_vp, _ip, _ip, _ll, _ip, _vp, _ip, _ip, _ip, _vp],
    "tpfnet_head": [_vp, _ll, _ip, _vp, _vp, _ip, _vp, _vp],
    "tpfnet_head_back": [_vp, _vp, _ll, _ip, _vp, _ip, _vp, _vp, _vp, _vp],
    "tpfnet_mse": [_vp, _vp, _vp, _ll, _ip, _vp, _vp, _vp],
    "tpfnet_adam": [_vp, _vp, _vp, _vp, _ll, _fl, _fl, _fl, _fl, _ip, _vp, _vp],
    "tpfnet_to_bf16": [_vp, _ll, _vp, _vp],
    "tpfnet_pack": [_vp, _vp, _ll, _ip, _ll, _vp, _vp, _vp, _ip, _ip, _vp],
    "tpfnet_unpack": [_vp, _ll, _ip, _vp, _vp, _vp, _vp, _ll, _vp],
}

PAD = 32  # channel granularity of the convolution kernels


def net_library():
    lib = load_library()
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    return lib


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def layer_specs(cin, cout, ch):
    """(name, Cin, Cout, taps) of every layer; Cin padded to the kernel granularity."""
    c0, c1, c2, c3 = ch
    cinp = -(-cin // PAD) * PAD
    spec = [("e0a", cinp, c0), ("e0b", c0, c0), ("e1a", c0, c1), ("e1b", c1, c1),
            ("e2a", c1, c2), ("e2b", c2, c2), ("b_a", c2, c3), ("b_b", c3, c3),
            ("d2a", c3 + c2, c2), ("d2b", c2, c2), ("d1a", c2 + c1, c1), ("d1b", c1, c1),
            ("d0a", c1 + c0, c0), ("d0b", c0, c0)]
    return [(n, a, b, 9) for n, a, b in spec] + [("head", c0, cout, 1)]


class UNet:
    def __init__(self, cin, cout, ch=(32, 64, 128, 256), seed=0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the U-Net kernels need a CUDA device")
        for c in ch:
            assert c % 64 == 0 or c == 32, "level channels: 32 or multiples of 64"
        self.torch = torch
        self.lib = net_library()
        self.cin, self.cout, self.ch = cin, cout, tuple(ch)
        self.cinp = -(-cin // PAD) * PAD
        self.specs = layer_specs(cin, cout, ch)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        rng = np.random.default_rng(seed)
        self.P, self.Pb, self.G, self.M, self.V = {}, {}, {}, {}, {}
        for name, a, b, taps in self.specs:
            fan_in = taps * (self.cin if name == "e0a" else a)
            w = rng.standard_normal((taps, b, a) if taps == 9 else (a, b)) * np.sqrt(2.0 / fan_in)
            if name == "e0a":
                w[:, :, cin:] = 0.0
            self._add(name + ".W", w.astype(np.float32), bf16=(taps == 9))
            self._add(name + ".b", (0.01 * rng.standard_normal(b)).astype(np.float32), bf16=False)
        self.adam_t = 0
        self._shape = None

    def _add(self, key, arr, bf16):
        t = self.torch
        self.P[key] = t.from_numpy(np.ascontiguousarray(arr)).cuda()
        self.G[key] = t.zeros_like(self.P[key])
        self.M[key] = t.zeros_like(self.P[key])
        self.V[key] = t.zeros_like(self.P[key])
        self.Pb[key] = self.P[key].to(t.bfloat16) if bf16 else None

    # ------------------------------------------------------- parameter I/O
    def set_reference_params(self, params):
        """Load parameters in the numpy reference layout (W[dh][dw][ci][co])."""
        for name, a, b, taps in self.specs:
            W = params[name + ".W"]
            if taps == 9:
                w = np.zeros((9, b, a), dtype=np.float32)
                w[:, :, :W.shape[2]] = W.reshape(9, W.shape[2], b).transpose(0, 2, 1)
            else:
                w = W.reshape(W.shape[2], b).astype(np.float32)
            self.P[name + ".W"].copy_(self.torch.from_numpy(w))
            if taps == 9:
                self.Pb[name + ".W"].copy_(self.P[name + ".W"].to(self.torch.bfloat16))
            self.P[name + ".b"].copy_(self.torch.from_numpy(params[name + ".b"].astype(np.float32)))

    def reference_grads(self):
        """Gradients in the numpy reference layout."""
        out = {}
        for name, a, b, taps in self.specs:
            g = self.G[name + ".W"].cpu().numpy().astype(np.float64)
            if taps == 9:
                ci = self.cin if name == "e0a" else a
                out[name + ".W"] = g.transpose(0, 2, 1)[:, :ci, :].reshape(3, 3, ci, b)
            else:
                out[name + ".W"] = g.reshape(1, 1, a, b)
            out[name + ".b"] = self.G[name + ".b"].cpu().numpy().astype(np.float64)
        return out

    def state_dict(self):
        return {k: v.cpu().numpy() for k, v in self.P.items()}

    def load_state_dict(self, d):
        for k, v in d.items():
            self.P[k].copy_(self.torch.from_numpy(v))
            if self.Pb[k] is not None:
                self.Pb[k].copy_(self.P[k].to(self.torch.bfloat16))

    # ---------------------------------------------------------- buffers
    def _buffers(self, N, H, W):
        if self._shape == (N, H, W):
            return
        assert H % 8 == 0 and W % 64 == 0, "H multiple of 8, W multiple of 64"
        t = self.torch
        c0, c1, c2, c3 = self.ch
        bf = dict(dtype=t.bfloat16, device="cuda")
        self.B = {}
        dims = [(H, W, c0), (H // 2, W // 2, c1), (H // 4, W // 4, c2), (H // 8, W // 8, c3)]
        for lvl, (h, w, c) in enumerate(dims):
            nm = ["e0", "e1", "e2", "b"][lvl]
            self.B[nm + "a"] = t.empty((N, h, w, c), **bf)
            self.B[nm] = t.empty((N, h, w, c), **bf)
            if lvl > 0:
                cin = dims[lvl - 1][2]
                self.B["pool%d" % lvl] = t.empty((N, h, w, cin), **bf)
        for lvl, (h, w, c) in ((2, dims[2]), (1, dims[1]), (0, dims[0])):
            cup = dims[lvl + 1][2] if lvl == 2 else self.ch[lvl + 1]
            self.B["cat%d" % lvl] = t.empty((N, h, w, cup + c), **bf)
            self.B["d%da" % lvl] = t.empty((N, h, w, c), **bf)
            self.B["d%d" % lvl] = t.empty((N, h, w, c), **bf)
        self.out = t.empty((N, H, W, self.cout), dtype=t.float32, device="cuda")
        # gradient buffers (one per activation shape)
        self.D = {k: t.empty_like(v) for k, v in self.B.items()}
        self.D["x"] = t.empty((N, H, W, self.cinp), **bf)
        self.D["out"] = t.empty_like(self.out)
        maxw = max(9 * a * b for _, a, b, taps in self.specs if taps == 9)
        self.wflip = t.empty(maxw, **bf)
        self.loss = t.zeros(1, dtype=t.float64, device="cuda")
        self._shape = (N, H, W)

    def _chk(self, rc, what):
        if rc != 0:
            raise RuntimeError("tpfnet kernel %s failed (%d)" % (what, rc))

    def _conv(self, name, x, N, H, W, cin, cout, y, relu=1):
        self._chk(self.lib.tpfnet_conv3x3(_p(x), N, H, W, cin, _p(self.Pb[name + ".W"]), _p(self.P[name + ".b"]),
                                          cout, relu, _p(y), self._s()), name)

    def _s(self):
        return C.c_void_p(self.stream.cuda_stream)

    # ---------------------------------------------------------- forward
    def forward(self, x):
        """x: bf16 CUDA tensor (N, H, W, cin padded to 32).  Returns float32 (N, H, W, cout)."""
        N, H, W, _ = x.shape
        self._buffers(N, H, W)
        self.x = x
        B, L = self.B, self.lib
        c0, c1, c2, c3 = self.ch
        s = self._s()
        dims = [(H, W), (H // 2, W // 2), (H // 4, W // 4), (H // 8, W // 8)]
        # encoder
        self._conv("e0a", x, N, H, W, self.cinp, c0, B["e0a"])
        self._conv("e0b", B["e0a"], N, H, W, c0, c0, B["e0"])
        prev, pc = B["e0"], c0
        for lvl, (nm, c) in enumerate((("e1", c1), ("e2", c2), ("b", c3)), start=1):
            h, w = dims[lvl]
            self._chk(L.tpfnet_pool(_p(prev), N, 2 * h, 2 * w, pc, _p(B["pool%d" % lvl]), s), "pool")
            ka, kb = ("b_a", "b_b") if nm == "b" else (nm + "a", nm + "b")
            self._conv(ka, B["pool%d" % lvl], N, h, w, pc, c, B[nm + "a"])
            self._conv(kb, B[nm + "a"], N, h, w, c, c, B[nm])
            prev, pc = B[nm], c
        # decoder
        skips = {2: (B["e2"], c2), 1: (B["e1"], c1), 0: (B["e0"], c0)}
        for lvl in (2, 1, 0):
            h, w = dims[lvl]
            skip, c = skips[lvl]
            cat = B["cat%d" % lvl]
            ctot = pc + c
            self._chk(L.tpfnet_up_into(_p(prev), N, h, w, pc, _p(cat), ctot, 0, s), "up")
            self._chk(L.tpfnet_channels(_p(skip), c, 0, N * h * w, c, _p(cat), ctot, pc, 0, s), "cat")
            self._conv("d%da" % lvl, cat, N, h, w, ctot, c, B["d%da" % lvl])
            self._conv("d%db" % lvl, B["d%da" % lvl], N, h, w, c, c, B["d%d" % lvl])
            prev, pc = B["d%d" % lvl], c
        self._chk(L.tpfnet_head(_p(prev), N * H * W, c0, _p(self.P["head.W"]), _p(self.P["head.b"]), self.cout,
                                _p(self.out), s), "head")
        return self.out

    # --------------------------------------------------------- backward
    def _block_back(self, ka, kb, inp, cin, a, bo, c, dout, dinp, N, h, w, need_dinp=True):
        """Back through relu(conv_b(relu(conv_a(inp)))): dout (grad at the block output,
        overwritten) -> weight grads and dinp."""
        L, s = self.lib, self._s()
        da = self.D["_tmp_%d_%d" % (h, c)]
        self._chk(L.tpfnet_relu_mask(_p(dout), _p(bo), dout.numel(), s), "mask")
        self._chk(L.tpfnet_conv3x3_wgrad(_p(a), _p(dout), N, h, w, c, c, _p(self.G[kb + ".W"]),
                                         _p(self.G[kb + ".b"]), s), "wgrad")
        self._chk(L.tpfnet_conv3x3_dgrad(_p(dout), N, h, w, c, _p(self.Pb[kb + ".W"]), c, _p(self.wflip), _p(da), s),
                  "dgrad")
        self._chk(L.tpfnet_relu_mask(_p(da), _p(a), da.numel(), s), "mask")
        self._chk(L.tpfnet_conv3x3_wgrad(_p(inp), _p(da), N, h, w, cin, c, _p(self.G[ka + ".W"]),
                                         _p(self.G[ka + ".b"]), s), "wgrad")
        if need_dinp:
            self._chk(L.tpfnet_conv3x3_dgrad(_p(da), N, h, w, c, _p(self.Pb[ka + ".W"]), cin, _p(self.wflip),
                                             _p(dinp), s), "dgrad")

    def backward(self, dout):
        """dout: float32 (N, H, W, cout) gradient of the loss at the output; accumulates
        every parameter gradient into self.G."""
        t, L, s = self.torch, self.lib, self._s()
        N, H, W = self._shape
        B, D = self.B, self.D
        c0, c1, c2, c3 = self.ch
        dims = [(H, W), (H // 2, W // 2), (H // 4, W // 4), (H // 8, W // 8)]
        for (h, w), c in zip(dims, self.ch):
            key = "_tmp_%d_%d" % (h, c)
            if key not in D:
                D[key] = t.empty((N, h, w, c), dtype=t.bfloat16, device="cuda")
        self._chk(L.tpfnet_head_back(_p(B["d0"]), _p(dout), N * H * W, c0, _p(self.P["head.W"]), self.cout,
                                     _p(D["d0"]), _p(self.G["head.W"]), _p(self.G["head.b"]), s), "head_back")
        skip_grads = {}
        # decoder levels 0, 1, 2: back through the block, split the concatenation
        ups = {0: c1, 1: c2, 2: c3}
        skips = {0: c0, 1: c1, 2: c2}
        below = {0: "d1", 1: "d2", 2: "b"}
        for lvl in (0, 1, 2):
            h, w = dims[lvl]
            cu, cs = ups[lvl], skips[lvl]
            ctot = cu + cs
            self._block_back("d%da" % lvl, "d%db" % lvl, B["cat%d" % lvl], ctot, B["d%da" % lvl], B["d%d" % lvl], cs,
                             D["d%d" % lvl], D["cat%d" % lvl], N, h, w)
            # the upsampled part goes to the level below, the skip part to the encoder
            self._chk(L.tpfnet_up_back(_p(D["cat%d" % lvl]), N, h, w, ctot, 0, cu, _p(D[below[lvl]]), s), "up_back")
            enc = ["e0", "e1", "e2"][lvl]
            self._chk(L.tpfnet_channels(_p(D["cat%d" % lvl]), ctot, cu, N * h * w, cs, _p(D[enc]), cs, 0, 0, s), "split")
        # bottleneck and encoder levels 2, 1, 0
        for lvl, nm, c in ((3, "b", c3), (2, "e2", c2), (1, "e1", c1)):
            h, w = dims[lvl]
            ka, kb = ("b_a", "b_b") if nm == "b" else (nm + "a", nm + "b")
            pc = self.ch[lvl - 1]
            self._block_back(ka, kb, B["pool%d" % lvl], pc, B[nm + "a"], B[nm], c, D[nm], D["pool%d" % lvl], N, h, w)
            enc_above = ["e0", "e1", "e2"][lvl - 1]
            self._chk(L.tpfnet_pool_back(_p(D["pool%d" % lvl]), N, 2 * h, 2 * w, pc, _p(D[enc_above]), 1, s), "pool_back")
        self._block_back("e0a", "e0b", self.x, self.cinp, B["e0a"], B["e0"], c0, D["e0"], D["x"], N, H, W,
                         need_dinp=False)

    def zero_grad(self):
        for g in self.G.values():
            g.zero_()

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.adam_t += 1
        s = self._s()
        for k, p in self.P.items():
            self._chk(self.lib.tpfnet_adam(_p(p), _p(self.G[k]), _p(self.M[k]), _p(self.V[k]), p.numel(), lr, b1, b2,
                                           eps, self.adam_t, _p(self.Pb[k]), s), "adam")

    def mse(self, pred, target, wch=None, want_grad=True):
        """Loss (float, synchronises) and, when want_grad, its gradient in self.D['out']."""
        self.loss.zero_()
        C_ = pred.shape[-1]
        self._chk(self.lib.tpfnet_mse(_p(pred), _p(target), _p(wch), pred.numel(), C_,
                                      _p(self.D["out"]) if want_grad else None, _p(self.loss), self._s()), "mse")
        return float(self.loss.item())

    def train_step(self, x, target, wch=None, lr=1e-3):
        self.zero_grad()
        out = self.forward(x)
        loss = self.mse(out, target, wch)
        self.backward(self.D["out"])
        self.adam(lr)
        return loss
