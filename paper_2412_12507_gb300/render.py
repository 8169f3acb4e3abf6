"""PyTorch-facing wrapper of the 3DGUT C ABI: device memory, streams and autograd.

PyTorch supplies device buffers and the current CUDA stream; every step of the hot path
(projection, binning / sorting, compositing, backward) runs in libut3d.so's kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import torch

from . import abi


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


@dataclass
class Scene:
    """Particle parameters as contiguous FP32 CUDA tensors (Sec. 3)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_arrays(d: dict, device="cuda") -> "Scene":
        f = lambda k: torch.as_tensor(d[k], dtype=torch.float32).contiguous().to(device)  # noqa: E731
        n = f("means").reshape(-1, 3).shape[0]
        deg = int(d["sh_degree"])
        return Scene(f("means").reshape(n, 3), f("log_scales").reshape(n, 3), f("quats").reshape(n, 4),
                     f("opacity_logits").reshape(n), f("sh").reshape(n, (deg + 1) ** 2, 3).contiguous(), deg)

    def struct(self) -> abi.UtScene:
        return abi.make_scene(self.means, self.log_scales, self.quats, self.opacity_logits, self.sh, self.sh_degree)


@dataclass
class Projection:
    mean2d: torch.Tensor
    cov2d: torch.Tensor
    depth: torch.Tensor
    rect: torch.Tensor
    ntiles: torch.Tensor


@dataclass
class Binning:
    vals: torch.Tensor
    ranges: torch.Tensor
    k_dev: torch.Tensor
    keys: torch.Tensor | None = None
    capacity: int = 0

    def count(self) -> int:
        return int(self.k_dev.item())


def project(scene: Scene, cam: dict, opts: dict | None = None, out: Projection | None = None) -> Projection:
    """ut_project: UT projection of every particle (Algorithms 1-2)."""
    n = scene.n
    dev = scene.means.device
    if out is None:
        out = Projection(torch.empty((n, 2), dtype=torch.float32, device=dev),
                         torch.empty((n, 3), dtype=torch.float32, device=dev),
                         torch.empty(n, dtype=torch.float32, device=dev),
                         torch.empty((n, 4), dtype=torch.int16, device=dev),
                         torch.empty(n, dtype=torch.int32, device=dev))
    c, o, u, s = abi.make_camera(cam), abi.make_options(opts), abi.make_params(opts), scene.struct()
    st = abi.lib().ut_project(C.byref(s), C.byref(c), C.byref(u), C.byref(o), _ptr(out.mean2d), _ptr(out.cov2d),
                              _ptr(out.depth), _ptr(out.rect), _ptr(out.ntiles), _stream())
    abi.check("ut_project", st)
    return out


def tile_count(cam: dict, opts: dict | None = None) -> int:
    o = abi.make_options(opts)
    return -(-int(cam["width"]) // o.tile_w) * -(-int(cam["height"]) // o.tile_h)


class Workspace:
    """Grow-only device scratch buffer (uint8), 256-byte aligned."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != torch.device(device):
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        p = self.buf.data_ptr()
        off = (-p) % 256
        return self.buf[off:off + nbytes]


def project_points(points: torch.Tensor, cam: dict, opts: dict | None = None):
    """ut_project_points: g of world points [n, 3] (float32, device) -> (uv [n, 2], valid [n] bool)."""
    pts = points.contiguous().float()
    n = pts.shape[0]
    uv = torch.empty((n, 2), dtype=torch.float32, device=pts.device)
    valid = torch.empty(n, dtype=torch.int32, device=pts.device)
    c, o = abi.make_camera(cam), abi.make_options(opts)
    abi.check("ut_project_points", abi.lib().ut_project_points(_ptr(pts), n, C.byref(c), C.byref(o), _ptr(uv),
                                                                _ptr(valid), _stream()))
    return uv, valid.bool()


def bin_and_sort(proj: Projection, cam: dict, opts: dict | None, capacity: int, want_keys: bool = False,
                 ws: Workspace | None = None, out: Binning | None = None) -> Binning:
    """bin_and_sort: duplicate (tile | depth) keys, stable sort, per-tile ranges (Sec. 4.3).

    Asynchronous: if the true key count exceeds `capacity`, out.count() reports it after the
    stream completes and the ranges are all empty (the caller retries)."""
    n = int(proj.depth.shape[0])
    dev = proj.depth.device
    c, o = abi.make_camera(cam), abi.make_options(opts)
    T = tile_count(cam, opts)
    capacity = int(max(capacity, 1))
    if out is None or out.capacity < capacity or (want_keys and out.keys is None):
        out = Binning(torch.empty(capacity, dtype=torch.int32, device=dev),
                      torch.empty((T, 2), dtype=torch.int32, device=dev),
                      torch.zeros(1, dtype=torch.int64, device=dev),
                      torch.empty(capacity, dtype=torch.int64, device=dev) if want_keys else None, capacity)
    ws = ws or Workspace()
    nbytes = abi.lib().ut_bin_workspace_size(n, out.capacity, C.byref(c), C.byref(o))
    w = ws.get(nbytes, dev)
    st = abi.lib().bin_and_sort(n, _ptr(proj.depth), _ptr(proj.rect), _ptr(proj.ntiles), C.byref(c), C.byref(o),
                                _ptr(w), w.numel(), out.capacity, _ptr(out.keys) if want_keys else None,
                                _ptr(out.vals), _ptr(out.ranges), _ptr(out.k_dev), _stream())
    abi.check("bin_and_sort", st)
    return out


@dataclass
class Frame:
    rgb: torch.Tensor
    alpha: torch.Tensor
    t_final: torch.Tensor
    n_used: torch.Tensor


def composite_forward(scene: Scene, cam: dict, opts: dict | None, proj: Projection, binning: Binning,
                      out: Frame | None = None, stats: torch.Tensor | None = None,
                      ws: Workspace | None = None) -> Frame:
    """composite_forward: front-to-back compositing with 3D max-response evaluation."""
    W, H = int(cam["width"]), int(cam["height"])
    dev = scene.means.device
    if out is None:
        out = Frame(torch.empty((3, H, W), dtype=torch.float32, device=dev),
                    torch.empty((H, W), dtype=torch.float32, device=dev),
                    torch.empty((H, W), dtype=torch.float32, device=dev),
                    torch.empty((H, W), dtype=torch.int32, device=dev))
    c, o, s = abi.make_camera(cam), abi.make_options(opts), scene.struct()
    ws = ws or Workspace()
    w = ws.get(abi.lib().ut_forward_workspace_size(C.byref(c), C.byref(o)), dev)
    st = abi.lib().composite_forward(C.byref(s), C.byref(c), C.byref(o), _ptr(proj.rect), _ptr(binning.vals),
                                     _ptr(binning.ranges), _ptr(out.rgb), _ptr(out.alpha), _ptr(out.t_final),
                                     _ptr(out.n_used), _ptr(w), w.numel(), _ptr(stats), _stream())
    abi.check("composite_forward", st)
    return out


def composite_backward(scene: Scene, cam: dict, opts: dict | None, proj: Projection, binning: Binning,
                       frame: Frame, d_rgb: torch.Tensor, d_alpha: torch.Tensor, ws: Workspace | None = None):
    """composite_backward: gradients of the loss w.r.t. every particle parameter."""
    n = scene.n
    dev = scene.means.device
    grads = dict(means=torch.empty_like(scene.means), log_scales=torch.empty_like(scene.log_scales),
                 quats=torch.empty_like(scene.quats), opacity_logits=torch.empty_like(scene.opacity_logits),
                 sh=torch.empty_like(scene.sh))
    ws = ws or Workspace()
    c, o, s = abi.make_camera(cam), abi.make_options(opts), scene.struct()
    w = ws.get(abi.lib().ut_backward_workspace_size(n, C.byref(c), C.byref(o)), dev)
    d_rgb = d_rgb.contiguous()
    d_alpha = d_alpha.contiguous()
    st = abi.lib().composite_backward(C.byref(s), C.byref(c), C.byref(o), _ptr(proj.rect), _ptr(binning.vals),
                                      _ptr(binning.ranges), _ptr(frame.rgb), _ptr(frame.t_final),
                                      _ptr(frame.n_used), _ptr(d_rgb), _ptr(d_alpha), _ptr(w), w.numel(),
                                      _ptr(grads["means"]), _ptr(grads["log_scales"]), _ptr(grads["quats"]),
                                      _ptr(grads["opacity_logits"]), _ptr(grads["sh"]), _stream())
    abi.check("composite_backward", st)
    return grads


@dataclass
class Renderer:
    """Renders one camera repeatedly, keeping workspaces and a key capacity that grows on demand."""
    cam: dict
    opts: dict | None = None
    capacity: int = 1 << 20
    growth: float = 1.25
    ws: Workspace = field(default_factory=Workspace)
    fws: Workspace = field(default_factory=Workspace)
    bws: Workspace = field(default_factory=Workspace)
    binning: Binning | None = None
    proj: Projection | None = None
    frame: Frame | None = None

    def forward(self, scene: Scene, sync_check: bool = True):
        self.proj = project(scene, self.cam, self.opts, self.proj if self.proj is not None and
                            self.proj.depth.shape[0] == scene.n else None)
        while True:
            self.binning = bin_and_sort(self.proj, self.cam, self.opts, self.capacity, ws=self.ws,
                                        out=self.binning)
            if not sync_check:
                break
            K = self.binning.count()
            if K <= self.binning.capacity:
                break
            self.capacity = int(K * self.growth) + 1
        self.frame = composite_forward(scene, self.cam, self.opts, self.proj, self.binning, self.frame, ws=self.fws)
        return self.frame

    def backward(self, scene: Scene, d_rgb: torch.Tensor, d_alpha: torch.Tensor):
        return composite_backward(scene, self.cam, self.opts, self.proj, self.binning, self.frame, d_rgb, d_alpha,
                                  self.bws)

    def capture(self, scene: Scene, d_rgb: torch.Tensor | None = None, d_alpha: torch.Tensor | None = None):
        """Records one forward step (and, given dL/drgb and dL/dalpha, one backward) on this
        renderer's current buffers as a CUDA graph; graph.replay() reruns every kernel of the step
        (projection, binning, compositing[, backward]) with no host launches.  Returns
        (graph, frame, grads or None): replays overwrite that frame and those gradient tensors.
        The key capacity is frozen into the graph: size it with a synchronised forward first
        (a replay whose key count exceeds it renders black and reports K in binning.k_dev)."""
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            self.forward(scene, sync_check=False)  # buffers exist before the capture
            if d_rgb is not None:
                self.backward(scene, d_rgb, d_alpha)
            stream.synchronize()
            with torch.cuda.graph(graph, stream=stream):
                frame = self.forward(scene, sync_check=False)
                grads = self.backward(scene, d_rgb, d_alpha) if d_rgb is not None else None
        torch.cuda.current_stream().wait_stream(stream)
        return graph, frame, grads


_SCENE_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


class FramePipeline:
    """Renders a stream of frames whose particle parameters arrive in host memory (pinned, for
    asynchronous copies), overlapping each frame's host-to-device copy and image read-back with
    the neighbouring frames' rendering.

    `depth` device copies of the scene, each with its own renderer (workspaces, frame) and its
    captured forward step, rotate: frame i's parameters are copied in on a copy stream while
    earlier frames render on the current stream, and each finished image is copied out on a
    read-back stream while the next frame renders; frame i's copy waits only for the read-back
    of frame i - depth.  `submit` returns the pinned [4][H][W] buffer (rgb, alpha) that
    receives the frame; it holds that frame once `done(buffer)` has been synchronised and until
    the submit `depth` frames later.  The key capacity is sized on the first frame (one
    synchronisation in the constructor); a later frame with more keys than it renders black
    (its count is in renderers[b].binning.k_dev)."""

    def __init__(self, cam: dict, opts: dict | None, first: dict, sh_degree: int, headroom: float = 1.25,
                 depth: int = 3):
        n = int(first["means"].numel() // 3)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.depth = int(depth)
        self.bufs = []
        for _ in range(self.depth):
            sc = Scene(torch.empty((n, 3), dtype=torch.float32, device=dev),
                       torch.empty((n, 3), dtype=torch.float32, device=dev),
                       torch.empty((n, 4), dtype=torch.float32, device=dev),
                       torch.empty(n, dtype=torch.float32, device=dev),
                       torch.empty((n, (sh_degree + 1) ** 2, 3), dtype=torch.float32, device=dev), sh_degree)
            for k in _SCENE_FIELDS:
                getattr(sc, k).copy_(first[k].view_as(getattr(sc, k)))
            self.bufs.append(sc)
        probe = Renderer(cam, opts)
        probe.forward(self.bufs[0])
        cap = int(probe.binning.count() * headroom) + 1024
        del probe
        self.renderers = [Renderer(cam, opts, capacity=cap) for _ in range(self.depth)]
        self.graphs = [r.capture(b)[:2] for r, b in zip(self.renderers, self.bufs)]
        H, W = int(cam["height"]), int(cam["width"])
        self.host_out = [torch.empty((4, H, W), dtype=torch.float32).pin_memory() for _ in range(self.depth)]
        self.copy_stream, self.read_stream = torch.cuda.Stream(), torch.cuda.Stream()
        self.copied = [torch.cuda.Event() for _ in range(self.depth)]
        self.rendered = [torch.cuda.Event() for _ in range(self.depth)]
        self.freed = [torch.cuda.Event() for _ in range(self.depth)]
        self.i = 0
        torch.cuda.synchronize()

    def submit(self, host: dict) -> torch.Tensor:
        b = self.i % self.depth
        self.i += 1
        sc, cs = self.bufs[b], torch.cuda.current_stream()
        self.copy_stream.wait_event(self.freed[b])  # frame i - depth no longer reads this buffer
        with torch.cuda.stream(self.copy_stream):
            for k in _SCENE_FIELDS:
                getattr(sc, k).copy_(host[k].view_as(getattr(sc, k)), non_blocking=True)
            self.copied[b].record(self.copy_stream)
        cs.wait_event(self.copied[b])
        graph, frame = self.graphs[b]
        graph.replay()
        self.rendered[b].record(cs)
        out = self.host_out[b]
        self.read_stream.wait_event(self.rendered[b])
        with torch.cuda.stream(self.read_stream):
            out[:3].copy_(frame.rgb, non_blocking=True)
            out[3].copy_(frame.alpha, non_blocking=True)
            self.freed[b].record(self.read_stream)
        return out

    def done(self, out: torch.Tensor) -> torch.cuda.Event:
        """The event after which `out` (a buffer submit returned) holds its frame."""
        return self.freed[next(i for i, h in enumerate(self.host_out) if h is out)]

    def join(self, stream: torch.cuda.Stream | None = None):
        """Makes `stream` (default: the current one) wait for every copy submitted so far."""
        s = stream or torch.cuda.current_stream()
        s.wait_stream(self.copy_stream)
        s.wait_stream(self.read_stream)


class RenderFunction(torch.autograd.Function):
    """torch.autograd.Function over the C ABI: (means, log_scales, quats, logits, sh) -> (rgb, alpha)."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, renderer: Renderer, sh_degree: int):
        scene = Scene(means.detach().contiguous(), log_scales.detach().contiguous(), quats.detach().contiguous(),
                      opacity_logits.detach().contiguous(), sh.detach().contiguous(), sh_degree)
        frame = renderer.forward(scene)
        ctx.renderer = renderer
        ctx.scene = scene
        ctx.proj, ctx.binning = renderer.proj, renderer.binning
        ctx.frame = Frame(frame.rgb.clone(), frame.alpha.clone(), frame.t_final.clone(), frame.n_used.clone())
        return ctx.frame.rgb.clone(), ctx.frame.alpha.clone()

    @staticmethod
    def backward(ctx, d_rgb, d_alpha):
        r = ctx.renderer
        if d_rgb is None:
            d_rgb = torch.zeros_like(ctx.frame.rgb)
        if d_alpha is None:
            d_alpha = torch.zeros_like(ctx.frame.alpha)
        g = composite_backward(ctx.scene, r.cam, r.opts, ctx.proj, ctx.binning, ctx.frame, d_rgb, d_alpha, r.bws)
        return g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], None, None


def render(means, log_scales, quats, opacity_logits, sh, sh_degree: int, renderer: Renderer):
    """Differentiable render through the C ABI; returns (rgb[3,H,W], alpha[H,W])."""
    return RenderFunction.apply(means, log_scales, quats, opacity_logits, sh, renderer, sh_degree)


# ---------------------------------------------------------------- batches of views

def _frame_for(cam: dict, dev, grad: bool) -> Frame:
    W, H = int(cam["width"]), int(cam["height"])
    return Frame(torch.empty((3, H, W), dtype=torch.float32, device=dev),
                 torch.empty((H, W), dtype=torch.float32, device=dev),
                 torch.empty((H, W), dtype=torch.float32, device=dev) if grad else None,
                 torch.empty((H, W), dtype=torch.int32, device=dev) if grad else None)


@dataclass
class BatchRenderer:
    """render_batch / render_batch_backward: several (scene, camera) views in one launch
    sequence.  views = list of (scene index, camera dict)."""
    scenes: list
    opts: dict | None = None
    capacity: int = 1 << 20
    growth: float = 1.25
    ws: Workspace = field(default_factory=Workspace)
    gws: Workspace = field(default_factory=Workspace)
    k_dev: torch.Tensor | None = None
    last: tuple | None = None

    def _structs(self, views, frames, d_rgb=None, d_alpha=None):
        sc = (abi.UtScene * len(self.scenes))(*[s.struct() for s in self.scenes])
        vw = (abi.UtView * len(views))()
        for j, ((si, cam), f) in enumerate(zip(views, frames)):
            v = vw[j]
            v.scene = int(si)
            v.camera = abi.make_camera(cam)
            v.rgb, v.alpha = _ptr(f.rgb), _ptr(f.alpha)
            v.t_final, v.n_used = _ptr(f.t_final), _ptr(f.n_used)
            if d_rgb is not None:
                v.d_rgb, v.d_alpha = _ptr(d_rgb[j]), _ptr(d_alpha[j])
        return sc, vw

    def forward(self, views, frames=None, grad: bool = False, sync_check: bool = True):
        """Renders every view; returns its Frame list (t_final / n_used kept when grad)."""
        dev = self.scenes[0].means.device
        if frames is None:
            frames = [_frame_for(cam, dev, grad) for _, cam in views]
        if self.k_dev is None:
            self.k_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        o, u = abi.make_options(self.opts), abi.make_params(self.opts)
        L = abi.lib()
        while True:
            sc, vw = self._structs(views, frames)
            nbytes = L.ut_batch_workspace_size(sc, len(self.scenes), vw, len(views), C.byref(o), self.capacity)
            if nbytes == 0:
                raise abi.UtError("ut_batch_workspace_size", abi.UT_ERR_INVALID_ARG, "invalid batch")
            w = self.ws.get(nbytes, dev)
            st = L.render_batch(sc, len(self.scenes), vw, len(views), C.byref(u), C.byref(o), _ptr(w), w.numel(),
                                self.capacity, _ptr(self.k_dev), _stream())
            abi.check("render_batch", st)
            if not sync_check:
                break
            K = int(self.k_dev.item())
            if K <= self.capacity:
                break
            self.capacity = int(K * self.growth) + 1
        self.last = (views, frames, w, self.capacity)
        return frames

    def backward(self, d_rgb, d_alpha):
        """Gradients of every scene for the views of the last forward; d_rgb / d_alpha: per view."""
        views, frames, w, cap = self.last
        dev = self.scenes[0].means.device
        d_rgb = [t.contiguous() for t in d_rgb]
        d_alpha = [t.contiguous() for t in d_alpha]
        grads = [dict(means=torch.empty_like(s.means), log_scales=torch.empty_like(s.log_scales),
                      quats=torch.empty_like(s.quats), opacity_logits=torch.empty_like(s.opacity_logits),
                      sh=torch.empty_like(s.sh)) for s in self.scenes]
        gs = (abi.UtSceneGrads * len(self.scenes))(*[
            abi.UtSceneGrads(_ptr(g["means"]), _ptr(g["log_scales"]), _ptr(g["quats"]), _ptr(g["opacity_logits"]),
                             _ptr(g["sh"])) for g in grads])
        sc, vw = self._structs(views, frames, d_rgb, d_alpha)
        L = abi.lib()
        o = abi.make_options(self.opts)
        gw = self.gws.get(L.ut_batch_backward_workspace_size(sc, len(self.scenes), vw, len(views), C.byref(o)), dev)
        st = L.render_batch_backward(sc, len(self.scenes), vw, len(views), C.byref(o), _ptr(w), w.numel(), cap,
                                     _ptr(gw), gw.numel(), gs, _stream())
        abi.check("render_batch_backward", st)
        return grads


class MultiViewRenderFunction(torch.autograd.Function):
    """One scene rendered from several cameras in one batch: (params) -> (rgb_0, alpha_0, rgb_1, ...)."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, renderer: BatchRenderer, cams, sh_degree: int):
        scene = Scene(means.detach().contiguous(), log_scales.detach().contiguous(), quats.detach().contiguous(),
                      opacity_logits.detach().contiguous(), sh.detach().contiguous(), sh_degree)
        renderer.scenes = [scene]
        views = [(0, c) for c in cams]
        frames = renderer.forward(views, grad=True)
        ctx.renderer = renderer
        out = []
        for f in frames:
            out += [f.rgb, f.alpha]
        return tuple(t.clone() for t in out)

    @staticmethod
    def backward(ctx, *grads):
        r = ctx.renderer
        views, frames = r.last[0], r.last[1]
        d_rgb = [g if g is not None else torch.zeros_like(f.rgb) for g, f in zip(grads[0::2], frames)]
        d_alpha = [g if g is not None else torch.zeros_like(f.alpha) for g, f in zip(grads[1::2], frames)]
        g = r.backward(d_rgb, d_alpha)[0]
        return g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], None, None, None


def render_views(means, log_scales, quats, opacity_logits, sh, sh_degree: int, cams, renderer: BatchRenderer):
    """Differentiable multi-view render of one scene in one batch; returns [(rgb, alpha)] per camera."""
    out = MultiViewRenderFunction.apply(means, log_scales, quats, opacity_logits, sh, renderer, cams, sh_degree)
    return [(out[2 * j], out[2 * j + 1]) for j in range(len(cams))]



TILE_CANDIDATES = ((8, 8), (16, 16), (32, 8), (16, 32))


def autotune_tiles(scenes: list, views, opts: dict | None = None, d_rgb=None, d_alpha=None,
                   candidates=TILE_CANDIDATES, steps: int = 3, warmup: int = 2):
    """Picks the tile shape for a batch of views by timing it: for every candidate
    (tile_w, tile_h) a BatchRenderer renders the batch (and, when d_rgb / d_alpha are given,
    runs its backward) `steps` times after `warmup` untimed runs, with CUDA events on the
    current stream.  Images do not depend on the tile shape (a pixel considers a particle iff
    its centre lies in the particle's rect), so only the speed differs.  Returns
    (best options dict, {"WxH": {"ms": per batch, "keys": K}})."""
    import copy
    base = dict(opts or {})
    results, best, best_ms = {}, None, float("inf")
    for tw, th in candidates:
        op = copy.deepcopy(base)
        op["tile_w"], op["tile_h"] = int(tw), int(th)
        br = BatchRenderer(scenes, op, capacity=1 << 20)
        grad = d_rgb is not None
        frames = br.forward(views, grad=grad)  # sizes the key capacity (synchronises)
        K = int(br.k_dev.item())

        def run():
            br.forward(views, frames=frames, grad=grad, sync_check=False)
            if grad:
                br.backward(d_rgb, d_alpha)

        for _ in range(warmup):
            run()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            run()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        results[f"{tw}x{th}"] = {"ms": ms, "keys": K}
        if ms < best_ms:
            best, best_ms = op, ms
        del br, frames
    return best, results

# ---------------------------------------------------------------- serving

class Server:
    """The library's request loop (ut_server_*): resident scenes, requests submitted from the
    host, admitted by the budget of a device arena, batched into render_batch launches on
    several streams.  Results are views into the arena, valid until released."""

    def __init__(self, scenes: list, opts: dict | None = None, arena_bytes: int = 1 << 32,
                 max_batch_views: int = 8, max_in_flight: int = 2, use_graphs: bool = True,
                 key_headroom: float = 1.3):
        self.scenes = scenes
        dev = scenes[0].means.device
        self.arena_buf = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device=dev)
        off = (-self.arena_buf.data_ptr()) % 256
        self.arena = self.arena_buf[off:off + int(arena_bytes)]
        cfg = abi.UtServerConfig(int(max_batch_views), int(max_in_flight), int(use_graphs), float(key_headroom),
                                 abi.make_options(opts), abi.make_params(opts))
        self._sc = (abi.UtScene * len(scenes))(*[s.struct() for s in scenes])
        h = C.c_void_p()
        torch.cuda.synchronize()  # scenes and arena must exist before the worker uses them
        abi.check("ut_server_create", abi.lib().ut_server_create(C.byref(cfg), self._sc, len(scenes),
                                                                 _ptr(self.arena), int(arena_bytes), C.byref(h)))
        self.h = h
        self.cams = {}

    def submit(self, scene: int, cam: dict) -> int:
        rid = C.c_uint64()
        c = abi.make_camera(cam)
        abi.check("ut_server_submit", abi.lib().ut_server_submit(self.h, int(scene), C.byref(c), C.byref(rid)))
        self.cams[rid.value] = cam
        return rid.value

    def wait(self, rid: int, timeout_ms: int = 10_000):
        """Returns (rgb[3,H,W], alpha[H,W], latency_ms) views into the arena, or None if not done."""
        done, rgb, alpha, lat = C.c_int32(), C.c_void_p(), C.c_void_p(), C.c_double()
        st = abi.lib().ut_server_wait(self.h, int(rid), int(timeout_ms), C.byref(done), C.byref(rgb),
                                      C.byref(alpha), C.byref(lat))
        if st == abi.UT_ERR_TIMEOUT:
            return None
        abi.check("ut_server_wait", st)
        if not done.value:
            return None
        cam = self.cams[rid]
        W, H = int(cam["width"]), int(cam["height"])
        base = self.arena.data_ptr()
        o = rgb.value - base
        img = self.arena[o:o + 16 * W * H].view(torch.float32)
        return img[:3 * W * H].view(3, H, W), img[3 * W * H:].view(H, W), lat.value

    def release(self, rid: int):
        abi.check("ut_server_release", abi.lib().ut_server_release(self.h, int(rid)))
        self.cams.pop(rid, None)

    def stats(self) -> dict:
        s = abi.UtServerStats()
        abi.check("ut_server_get_stats", abi.lib().ut_server_get_stats(self.h, C.byref(s)))
        return {k: int(getattr(s, k)) for k, _ in abi.UtServerStats._fields_}

    def close(self):
        if self.h:
            abi.check("ut_server_destroy", abi.lib().ut_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
