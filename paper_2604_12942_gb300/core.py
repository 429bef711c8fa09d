"""Python binding of libgs.so (include/gs.h) over PyTorch device memory and streams.

Marshalling only: tensors become device pointers, camera dicts become gs_camera structs,
and each method calls one C entry point on the current CUDA stream.  The mapping step of
RMGS-SLAM §III-C (projection, tile sort, compositing of colour and depth, L1 loss, analytic
backward incl. pose twists, masked Adam) runs entirely in the library's kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as N

PARAM_GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def n_planes(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


def default_opts(**kw) -> N.RenderOpts:
    o = N.RenderOpts()
    N.lib().gs_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "bg":
            o.bg = (C.c_float * 3)(*v)
        else:
            setattr(o, k, v)
    return o


def camera_array(cams) -> C.Array:
    arr = (N.Camera * len(cams))()
    for c, d in zip(arr, cams):
        c.width, c.height = int(d["width"]), int(d["height"])
        c.fx, c.fy, c.cx, c.cy = float(d["fx"]), float(d["fy"]), float(d["cx"]), float(d["cy"])
        c.R_cw = (C.c_float * 9)(*np.asarray(d["R"], dtype=np.float64).reshape(-1).tolist())
        c.t_cw = (C.c_float * 3)(*np.asarray(d["t"], dtype=np.float64).reshape(-1).tolist())
    return arr


def gaussians_struct(planes: torch.Tensor, sh_degree: int) -> N.Gaussians:
    """gs_gaussians pointing into a packed [11 + 3K, n] float32 CUDA tensor."""
    assert planes.is_cuda and planes.dtype == torch.float32 and planes.is_contiguous()
    P, n = planes.shape
    assert P == n_planes(sh_degree), (P, sh_degree)
    base = planes.data_ptr()
    row = 4 * n
    return N.Gaussians(n, sh_degree, base, base + 3 * row, base + 6 * row, base + 10 * row, base + 11 * row)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def pixel_offsets(cams):
    off = [0]
    for c in cams:
        off.append(off[-1] + int(c["width"]) * int(c["height"]))
    return off


def pack_rgb(images, device="cuda") -> torch.Tensor:
    """Per-view [3, H, W] arrays -> the packed planar colour buffer of gs.h."""
    return torch.cat([torch.as_tensor(np.ascontiguousarray(im), dtype=torch.float32).reshape(-1)
                      for im in images]).to(device)


def pack_plane(planes, dtype=torch.float32, device="cuda") -> torch.Tensor:
    return torch.cat([torch.as_tensor(np.ascontiguousarray(p)).to(dtype).reshape(-1) for p in planes]).to(device)


def unpack_rgb(buf: torch.Tensor, cams):
    off = pixel_offsets(cams)
    return [buf[3 * off[v]:3 * off[v + 1]].reshape(3, c["height"], c["width"]) for v, c in enumerate(cams)]


def unpack_plane(buf: torch.Tensor, cams):
    off = pixel_offsets(cams)
    return [buf[off[v]:off[v + 1]].reshape(c["height"], c["width"]) for v, c in enumerate(cams)]


class Workspace:
    """A device workspace laid out for (n Gaussians, these cameras' image sizes, tile,
    max_pairs) plus the host-side gs_ws_layout descriptor."""

    def __init__(self, n, cams, opts: N.RenderOpts, max_pairs, device="cuda"):
        self.cams_c = camera_array(cams)
        self.cams = cams
        self.opts = opts
        self.layout = N.WsLayout()
        N.check(N.lib().gs_workspace_layout(int(n), len(cams), self.cams_c, C.byref(opts), int(max_pairs),
                                            C.byref(self.layout)), "gs_workspace_layout")
        self.buf = torch.empty(int(self.layout.total), dtype=torch.uint8, device=device)
        assert self.buf.data_ptr() % 256 == 0
        self.n = int(n)
        self.V = len(cams)
        N.check(N.lib().gs_workspace_init(C.byref(self.layout), _ptr(self.buf), _stream()), "gs_workspace_init")

    def set_cameras(self, cams):
        """New poses (same image sizes) for the next calls."""
        self.cams_c = camera_array(cams)
        self.cams = cams

    def region(self, name, dtype, count):
        off = getattr(self.layout, name)
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        return self.buf[off:off + nbytes].view(dtype)

    # -- stage calls -----------------------------------------------------------------------
    def project(self, planes, sh_degree):
        g = gaussians_struct(planes, sh_degree)
        N.check(N.lib().gs_project(C.byref(g), self.cams_c, C.byref(self.opts), C.byref(self.layout),
                                   _ptr(self.buf), _stream()), "gs_project")

    def bin_sort(self):
        N.check(N.lib().gs_bin_sort(self.cams_c, C.byref(self.opts), C.byref(self.layout), _ptr(self.buf), _stream()),
                "gs_bin_sort")

    def render_fwd(self, out_rgb, out_depth, out_T=None, target_rgb=None, target_depth=None, mask=None,
                   dl_drgb=None, dl_ddepth=None, loss_out=None):
        N.check(N.lib().gs_render_fwd(self.cams_c, C.byref(self.opts), C.byref(self.layout), _ptr(self.buf),
                                      _ptr(out_rgb), _ptr(out_depth), _ptr(out_T), _ptr(target_rgb),
                                      _ptr(target_depth), _ptr(mask), _ptr(dl_drgb), _ptr(dl_ddepth),
                                      _ptr(loss_out), _stream()), "gs_render_fwd")

    def render_mask(self, mask_out, caller_mask=None):
        """Interior mask of the last forward's transmittance (opts.mask_opacity, mask_erode)."""
        N.check(N.lib().gs_render_mask(self.cams_c, C.byref(self.opts), C.byref(self.layout), _ptr(self.buf),
                                       _ptr(caller_mask), _ptr(mask_out), _stream()), "gs_render_mask")

    def objective(self, rgb, depth, target_rgb, target_depth, mask, dl_drgb, dl_ddepth, loss_out):
        """lambda_rgb L_rgb + lambda_ssim (1 - SSIM) + lambda_depth L_depth over `mask`, with
        dL/dC and dL/dD."""
        N.check(N.lib().gs_objective(self.cams_c, C.byref(self.opts), C.byref(self.layout), _ptr(self.buf),
                                     _ptr(rgb), _ptr(depth), _ptr(target_rgb), _ptr(target_depth), _ptr(mask),
                                     _ptr(dl_drgb), _ptr(dl_ddepth), _ptr(loss_out), _stream()), "gs_objective")

    def render_bwd(self, planes, sh_degree, grad_planes, dl_drgb, dl_ddepth=None, grad_twist=None):
        g = gaussians_struct(planes, sh_degree)
        gg = gaussians_struct(grad_planes, sh_degree)
        N.check(N.lib().gs_render_bwd(C.byref(g), self.cams_c, C.byref(self.opts), C.byref(self.layout),
                                      _ptr(self.buf), _ptr(dl_drgb), _ptr(dl_ddepth), C.byref(gg),
                                      _ptr(grad_twist), _stream()), "gs_render_bwd")

    def composite_bwd(self, dl_drgb, dl_ddepth=None):
        N.check(N.lib().gs_composite_bwd(self.cams_c, C.byref(self.opts), C.byref(self.layout), _ptr(self.buf),
                                         _ptr(dl_drgb), _ptr(dl_ddepth), _stream()), "gs_composite_bwd")

    def project_bwd(self, planes, sh_degree, grad_planes, grad_twist=None):
        g = gaussians_struct(planes, sh_degree)
        gg = gaussians_struct(grad_planes, sh_degree)
        N.check(N.lib().gs_project_bwd(C.byref(g), self.cams_c, C.byref(self.opts), C.byref(self.layout),
                                       _ptr(self.buf), C.byref(gg), _ptr(grad_twist), _stream()), "gs_project_bwd")

    def project_bwd_adam(self, planes, sh_degree, m, v, step, lr, update_mask=None, b1=0.9, b2=0.999, eps=1e-15,
                         grad_twist=None):
        """Fused projection backward + masked Adam (parameters, m, v updated in place)."""
        gp, gm, gv = (gaussians_struct(t, sh_degree) for t in (planes, m, v))
        lrs = (C.c_float * 6)(*lr)
        N.check(N.lib().gs_project_bwd_adam(C.byref(gp), self.cams_c, C.byref(self.opts), C.byref(self.layout),
                                            _ptr(self.buf), C.byref(gm), C.byref(gv), _ptr(update_mask), lrs, b1, b2,
                                            eps, int(step), _ptr(grad_twist), _stream()), "gs_project_bwd_adam")

    def counters(self) -> N.Counters:
        c = N.Counters()
        N.check(N.lib().gs_read_counters(C.byref(self.layout), _ptr(self.buf), C.byref(c), _stream()),
                "gs_read_counters")
        return c

    # -- views of intermediate state (for tests) ------------------------------------------
    def sorted_pairs(self, n_pairs):
        """The sorted pairs as (key, value) with key = (tile id << 32) | bits(z) -- the tile
        ids from the sort's output, z from each value's projected record."""
        L = self.layout
        kname, vname = ("keys1", "vals1") if L.sorted_buf else ("keys0", "vals0")
        tiles = self.region(kname, torch.int32, n_pairs).to(torch.int64) & 0xFFFFFFFF
        vals = self.region(vname, torch.int32, n_pairs)
        rec = self.region("proj", torch.int32, 12 * self.layout.n_views * self.n)
        zbits = rec[vals.to(torch.int64) * 12 + 2].to(torch.int64) & 0xFFFFFFFF
        return (tiles << 32) | zbits, vals

    def sorted_entries(self, n_entries):
        """The visible (view, Gaussian) entries in depth order (values view * n + index)."""
        order = self.region("evals0", torch.int32, n_entries).to(torch.int64)
        return self.region("entries", torch.int32, n_entries)[order]

    def visible(self):
        return self.region("visible", torch.uint8, self.n)


class Renderer:
    """Differentiable rendering of the Gaussian map into a batch of keyframes (§III-C: colour
    and depth composited front to back; gradients to every Gaussian parameter and to each
    keyframe pose), usable inside any PyTorch computation:

        r = Renderer(n, cams, sh_degree)
        rgb, depth, T = r(planes, twist)          # RenderFn.apply(planes, twist, r)
        loss = my_objective(rgb, depth)
        loss.backward()                           # planes.grad, twist.grad

    `planes` is the packed [11 + 3K, n] float32 CUDA tensor of gs.h (means, log-scales,
    quaternions, opacity logit, SH).  `twist` (may be None) is a [V, 6] float32 tensor on any
    device: pose increments xi = (rho, phi) applied on the left, T_cw <- Exp(xi) T_cw, to the
    cameras given here; its gradient is the exact gradient w.r.t. xi.  The outputs are the
    packed images of gs.h (rgb [3P] planar per view, depth [P], final transmittance T [P];
    unpack with unpack_rgb / unpack_plane); T carries no gradient.

    The forward reads the twist on the host and checks the workspace's status word (both
    synchronise the stream); the backward reads the pose gradient back the same way.  One
    workspace holds the state of one forward: a second forward through the same Renderer
    before the first one's backward makes that backward raise."""

    def __init__(self, n, cams, sh_degree, opts: N.RenderOpts | None = None, max_pairs=None, device="cuda"):
        self.ws = Workspace(n, cams, opts or default_opts(), max_pairs or max(1 << 20, 64 * n * len(cams)), device)
        self.base_cams = camera_array(cams)
        self.sh_degree = sh_degree
        self.generation = 0

    def __call__(self, planes, twist=None):
        return RenderFn.apply(planes, twist, self)


class RenderFn(torch.autograd.Function):
    """forward: gs_twist_cameras (if a twist is given), gs_project, gs_bin_sort, gs_render_fwd;
    backward: gs_render_bwd for the upstream dL/dC, dL/dD, then gs_twist_grad for the poses.
    Marshalling only: every step runs in the library."""

    @staticmethod
    def forward(ctx, planes, twist, r: Renderer):
        ws = r.ws
        V = ws.V
        xi = None
        cams = r.base_cams
        if twist is not None:
            if tuple(twist.shape) != (V, 6):
                raise ValueError(f"twist must be [{V}, 6], got {tuple(twist.shape)}")
            xi = twist.detach().to("cpu", torch.float32).contiguous()
            cams = (N.Camera * V)()
            N.check(N.lib().gs_twist_cameras(r.base_cams, C.c_void_p(xi.data_ptr()), V, cams), "gs_twist_cameras")
        ws.cams_c = cams
        P = ws.layout.total_pixels
        dev = planes.device
        rgb = torch.empty(3 * P, device=dev)
        depth = torch.empty(P, device=dev)
        T = torch.empty(P, device=dev)
        ws.project(planes, r.sh_degree)
        ws.bin_sort()
        ws.render_fwd(rgb, depth, T)
        c = ws.counters()
        if c.status != 0:
            raise N.GsError(f"render: device status {N.STATUS.get(c.status, c.status)} ({c.n_pairs} pairs for "
                            f"a workspace of {ws.layout.max_pairs}); make the Renderer with a larger max_pairs")
        r.generation += 1
        ctx.generation = r.generation
        ctx.r, ctx.cams, ctx.xi = r, cams, xi
        ctx.twist_device = None if twist is None else twist.device
        ctx.save_for_backward(planes)
        ctx.mark_non_differentiable(T)
        return rgb, depth, T

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_T):
        r = ctx.r
        if r.generation != ctx.generation:
            raise RuntimeError("RenderFn.backward: the Renderer's workspace was used by a later forward; "
                               "use one Renderer per forward whose backward is still pending")
        (planes,) = ctx.saved_tensors
        ws = r.ws
        ws.cams_c = ctx.cams
        V = ws.V
        P = ws.layout.total_pixels
        dev = planes.device
        want_twist = ctx.xi is not None and ctx.needs_input_grad[1]
        grads = torch.zeros_like(planes)
        g_left = torch.zeros(V, 6, device=dev) if want_twist else None
        g_rgb = torch.zeros(3 * P, device=dev) if g_rgb is None else g_rgb.contiguous().to(torch.float32)
        g_depth = None if g_depth is None else g_depth.contiguous().to(torch.float32)
        ws.render_bwd(planes, r.sh_degree, grads, g_rgb, g_depth, g_left)
        g_xi = None
        if want_twist:
            gl = g_left.cpu()
            gx = torch.empty(V, 6)
            N.check(N.lib().gs_twist_grad(C.c_void_p(ctx.xi.data_ptr()), C.c_void_p(gl.data_ptr()), V,
                                          C.c_void_p(gx.data_ptr())), "gs_twist_grad")
            g_xi = gx.to(ctx.twist_device)
        return (grads if ctx.needs_input_grad[0] else None), g_xi, None


def adam_step(planes, grads, m, v, sh_degree, step, lr, update_mask=None, visible=None, b1=0.9, b2=0.999,
              eps=1e-15):
    gp, gg, gm, gv = (gaussians_struct(t, sh_degree) for t in (planes, grads, m, v))
    lrs = (C.c_float * 6)(*lr)
    N.check(N.lib().gs_adam_step(C.byref(gp), C.byref(gg), C.byref(gm), C.byref(gv), _ptr(update_mask),
                                 _ptr(visible), lrs, b1, b2, eps, int(step), _stream()), "gs_adam_step")


LR_DEFAULT = (1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4)


@dataclass
class StepResult:
    loss: torch.Tensor          # [V + 1] device: per-view terms and their mean
    rgb: torch.Tensor
    depth: torch.Tensor


class MappingStep:
    """One optimisation step of the Gaussian map over a batch of keyframes (gs_step): project,
    tile sort, composite with the fused L1 loss, backward (with pose twists) and masked Adam,
    all views of the batch in each launch, one C call.  `capture()` records the step as a
    CUDA graph (gs_graph_create) and `replay()` launches it; `set_cameras()` changes the
    poses of a captured graph without re-capturing."""

    def __init__(self, planes: torch.Tensor, sh_degree: int, cams, opts: N.RenderOpts | None = None,
                 max_pairs: int | None = None, lr=LR_DEFAULT, b1=0.9, b2=0.999, eps=1e-15):
        self.planes = planes
        self.sh_degree = sh_degree
        self.opts = opts or default_opts()
        n = planes.shape[1]
        self.ws = Workspace(n, cams, self.opts, max_pairs or max(1 << 20, 64 * n * len(cams)), planes.device)
        P = self.ws.layout.total_pixels
        dev = planes.device
        self.grads = torch.zeros_like(planes)
        self.m = torch.zeros_like(planes)
        self.v = torch.zeros_like(planes)
        self.rgb = torch.empty(3 * P, device=dev)
        self.depth = torch.empty(P, device=dev)
        self.dl_drgb = torch.empty(3 * P, device=dev)
        self.dl_ddepth = torch.empty(P, device=dev)
        self.loss = torch.zeros(len(cams) + 1, device=dev)
        self.twist = torch.zeros(len(cams), 6, device=dev)
        self.lr, self.b1, self.b2, self.eps = tuple(lr), b1, b2, eps
        self._structs = [gaussians_struct(t, sh_degree) for t in (self.planes, self.grads, self.m, self.v)]
        self.graph = None
        self._graph_io = None

    def _io(self, target_rgb, target_depth, mask, update_mask, optimize, with_twist, host=None):
        io = N.StepIO()
        if host is not None:
            # pinned host buffers (rgb, depth, mask, loss), each may be None: the step copies the
            # targets from them into the device buffers above and the loss back
            for name, t in zip(("host_target_rgb", "host_target_depth", "host_mask", "host_loss_out"), host):
                if t is not None:
                    assert not t.is_cuda and t.is_pinned() and t.is_contiguous(), name
                    setattr(io, name, t.data_ptr())
        io.target_rgb, io.target_depth = target_rgb.data_ptr(), (target_depth.data_ptr() if target_depth is not None else None)
        io.mask = mask.data_ptr() if mask is not None else None
        io.out_rgb, io.out_depth = self.rgb.data_ptr(), self.depth.data_ptr()
        io.dl_drgb, io.dl_ddepth = self.dl_drgb.data_ptr(), self.dl_ddepth.data_ptr()
        io.loss_out = self.loss.data_ptr()
        io.grad_twist = self.twist.data_ptr() if with_twist else None
        io.update_mask = update_mask.data_ptr() if update_mask is not None else None
        io.lr = (C.c_float * 6)(*self.lr)
        io.b1, io.b2, io.eps = self.b1, self.b2, self.eps
        io.optimize = 1 if optimize else 0
        return io

    def __call__(self, target_rgb, target_depth=None, mask=None, update_mask=None, optimize=True,
                 with_twist=False, host=None) -> StepResult:
        io = self._io(target_rgb, target_depth, mask, update_mask, optimize, with_twist, host)
        gp, gg, gm, gv = self._structs
        N.check(N.lib().gs_step(C.byref(gp), C.byref(gg), C.byref(gm), C.byref(gv), self.ws.cams_c,
                                C.byref(self.opts), C.byref(self.ws.layout), _ptr(self.ws.buf), C.byref(io), _stream()),
                "gs_step")
        return StepResult(self.loss, self.rgb, self.depth)

    def capture(self, target_rgb, target_depth=None, mask=None, update_mask=None, optimize=True, with_twist=False,
                host=None):
        """Record one step as a CUDA graph (inputs are read from these buffers at replay).  With
        host = (pinned rgb, depth, mask, loss) tensors (any may be None) every replay uploads
        the targets from host memory (overlapped with the projection and binning) and copies
        the loss back to host memory."""
        self.release()
        io = self._io(target_rgb, target_depth, mask, update_mask, optimize, with_twist, host)
        self._graph_io = (io, target_rgb, target_depth, mask, update_mask, host)
        side = torch.cuda.Stream(device=self.planes.device)
        side.wait_stream(torch.cuda.current_stream())
        h = C.c_void_p()
        gp, gg, gm, gv = self._structs
        N.check(N.lib().gs_graph_create(C.byref(h), C.byref(gp), C.byref(gg), C.byref(gm), C.byref(gv),
                                        self.ws.cams_c, C.byref(self.opts), C.byref(self.ws.layout), _ptr(self.ws.buf),
                                        C.byref(io), C.c_void_p(side.cuda_stream)), "gs_graph_create")
        torch.cuda.current_stream().wait_stream(side)
        self.graph = h

    def replay(self) -> StepResult:
        N.check(N.lib().gs_graph_launch(self.graph, _stream()), "gs_graph_launch")
        return StepResult(self.loss, self.rgb, self.depth)

    def set_cameras(self, cams):
        """New poses (same image sizes) for the eager step and for a captured graph."""
        self.ws.set_cameras(cams)
        if self.graph is not None:
            N.check(N.lib().gs_graph_set_cameras(self.graph, self.ws.cams_c), "gs_graph_set_cameras")

    def release(self):
        if self.graph is not None:
            N.lib().gs_graph_destroy(self.graph)
            self.graph = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


# -- map-size updates between mapping iterations (f2) -----------------------------------------
def map_update_scratch(n_map, n_new=0, device="cuda") -> torch.Tensor:
    return torch.empty(int(N.lib().gs_map_update_scratch_bytes(int(n_map), int(n_new))), dtype=torch.uint8,
                       device=device)


def prune_plan(planes, sh_degree, opacity_min=0.005, max_ratio=0.01, scratch=None):
    """(keep uint8 [n], rows kept): low-opacity rows to remove, at most max_ratio of the map."""
    n = planes.shape[1]
    keep = torch.empty(n, dtype=torch.uint8, device=planes.device)
    scratch = map_update_scratch(n, 0, planes.device) if scratch is None else scratch
    nk = C.c_int64()
    g = gaussians_struct(planes, sh_degree)
    N.check(N.lib().gs_prune_plan(C.byref(g), float(opacity_min), float(max_ratio), _ptr(keep), _ptr(scratch),
                                  scratch.numel(), C.byref(nk), _stream()), "gs_prune_plan")
    return keep, nk.value


def dedup_plan(planes, sh_degree, new_means, radius=0.05, scratch=None):
    """(accept uint8 [n_new], accepted): new means [3, n_new] with no map mean within radius."""
    new_means = new_means.contiguous()
    n_new = new_means.shape[1]
    accept = torch.empty(max(n_new, 1), dtype=torch.uint8, device=planes.device)[:n_new]
    scratch = map_update_scratch(planes.shape[1], n_new, planes.device) if scratch is None else scratch
    na = C.c_int64()
    g = gaussians_struct(planes, sh_degree)
    N.check(N.lib().gs_dedup_plan(C.byref(g), _ptr(new_means), n_new, float(radius), _ptr(accept), _ptr(scratch),
                                  scratch.numel(), C.byref(na), _stream()), "gs_dedup_plan")
    return accept, na.value


def map_update(planes, m, v, sh_degree, keep, new_planes=None, accept=None, tags=None, new_tags=None,
               scratch=None):
    """New (planes, m, v[, tags]) tensors: kept rows in order, then accepted new rows (zero
    moments)."""
    n = planes.shape[1]
    n_new = 0 if new_planes is None else new_planes.shape[1]
    n_out = int(keep.sum()) + (0 if new_planes is None else (n_new if accept is None else int(accept.sum())))
    P = planes.shape[0]
    dev = planes.device
    out, m_out, v_out = (torch.empty(P, n_out, device=dev) for _ in range(3))
    tags_out = torch.empty(n_out, dtype=torch.int32, device=dev) if tags is not None else None
    scratch = map_update_scratch(n, n_new, dev) if scratch is None else scratch
    gs_ = [gaussians_struct(t, sh_degree) for t in (planes, m, v)]
    go = [gaussians_struct(t, sh_degree) for t in (out, m_out, v_out)]
    gn = gaussians_struct(new_planes.contiguous(), sh_degree) if new_planes is not None else None
    N.check(N.lib().gs_map_update(C.byref(gs_[0]), C.byref(gs_[1]), C.byref(gs_[2]), _ptr(keep),
                                  C.byref(gn) if gn is not None else None, _ptr(accept), _ptr(tags), _ptr(new_tags),
                                  C.byref(go[0]), C.byref(go[1]), C.byref(go[2]), _ptr(tags_out), _ptr(scratch),
                                  scratch.numel(), _stream()), "gs_map_update")
    return (out, m_out, v_out) if tags is None else (out, m_out, v_out, tags_out)


# -- Gaussian-GICP loop registration (f3) -------------------------------------------------------
def gicp_target_set(planes, sh_degree, cams, near_z=0.2, d_max=20.0, source_flag=None, scratch=None):
    """(target_flag uint8 [n], count): map rows seen by some query view, within d_max of it,
    outside the source set."""
    n = planes.shape[1]
    flag = torch.empty(max(n, 1), dtype=torch.uint8, device=planes.device)[:n]
    scratch = gicp_scratch(0, planes.device) if scratch is None else scratch
    cnt = C.c_int64()
    g = gaussians_struct(planes, sh_degree)
    N.check(N.lib().gs_gicp_target_set(C.byref(g), camera_array(cams), len(cams), float(near_z), float(d_max),
                                       _ptr(source_flag), _ptr(flag), _ptr(scratch), scratch.numel(), C.byref(cnt),
                                       _stream()), "gs_gicp_target_set")
    return flag, cnt.value


def gicp_scratch(n_target_map, device="cuda") -> torch.Tensor:
    return torch.empty(int(N.lib().gs_gicp_scratch_bytes(int(n_target_map))), dtype=torch.uint8, device=device)


def gicp_register(src_planes, src_flag, tar_planes, tar_flag, sh_degree, T_init=None, d_corr=1.0, max_iters=30,
                  eps=1e-7, scratch=None):
    """Loop transform (4 x 4 numpy) mapping the source rows onto the target rows, and the
    result record (cost, correspondences, iterations, converged)."""
    import numpy as np
    T0 = np.eye(4) if T_init is None else np.asarray(T_init, dtype=np.float64)
    t12 = (C.c_double * 12)(*T0[:3, :4].reshape(-1).tolist())
    scratch = gicp_scratch(tar_planes.shape[1], tar_planes.device) if scratch is None else scratch
    res = N.GicpResult()
    gs_ = gaussians_struct(src_planes, sh_degree)
    gt = gaussians_struct(tar_planes, sh_degree)
    N.check(N.lib().gs_gicp_register(C.byref(gs_), _ptr(src_flag), C.byref(gt), _ptr(tar_flag), t12, float(d_corr),
                                     int(max_iters), float(eps), C.byref(res), _ptr(scratch), scratch.numel(),
                                     _stream()), "gs_gicp_register")
    T = np.eye(4)
    T[:3, :4] = np.array(list(res.T)).reshape(3, 4)
    return T, res

