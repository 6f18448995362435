"""The optimisation step (rows a1-a10) for one lens or a batch of lenses.

One step = forward trace -> loss and dL/dE -> recompute adjoint -> Adam, all on
one stream. With graph=True the step is captured once into a CUDA graph and
every later step is one graph replay. The control heights, Adam moments and the
step counter of all lenses live in flat device buffers, so one Adam launch
updates every lens.

loss="l2" is the squared L2 distance to the target; loss="frobenius" the
paper's normalised Frobenius loss (Sec. 2.5). With reparam=dict(z_min=...,
z_max=..., offset=...) Adam runs on unconstrained variables theta and the
control heights are P = offset + z_min + (tanh(theta) + 1)(z_max - z_min)/2
(Sec. 2.4.2); offset is None, a ("sphere", c, R) cap of Table magndata, or an
array per lens. The fused Adam kernel writes P from the new theta.
"""
import numpy as np
import torch

from . import api


class OptimStep:
    def __init__(self, workloads, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, options=None, graph=True,
                 device="cuda", adj_options=None, loss="l2", reparam=None, pdl=True, ray_order=True):
        """`options` apply to both traces unless `adj_options` is given for the adjoint
        (e.g. to record timing events around each trace kernel separately).
        ray_order: point-source lenses trace their rays
        in the coherent order of fr_ray_order (built once here, from the starting
        heights' mean: any order gives the same sums, so it stays valid as the
        heights move)."""
        if isinstance(workloads, dict):
            workloads = [workloads]
        if loss not in ("l2", "frobenius"):
            raise ValueError("loss must be 'l2' or 'frobenius'")
        self.loss_kind = loss
        self.reparam = reparam
        self.pdl = pdl   # programmatic dependent launch between the step's kernels
        self.h = api.default_handle()
        self.lr, self.betas, self.eps = lr, betas, eps
        self.options = options
        self.adj_options = adj_options if adj_options is not None else options
        # The step clears E and dL/dP itself (memsets first), so that the
        # trace calls accumulate and the four kernels follow one another
        # directly: with programmatic launch each may start while the previous
        # one drains.
        self._fwd_opts = self._accumulating(self.options)
        self._adj_opts = self._accumulating(self.adj_options)
        # per lens: the exit heights, then (two-face lenses) the entry heights
        n_out = [(w["lens"]["n1"] + 1) * (w["lens"]["n2"] + 1) for w in workloads]
        n_in = [(w["lens"]["n1_in"] + 1) * (w["lens"]["n2_in"] + 1) if w["lens"].get("P_in") is not None else 0
                for w in workloads]
        sizes = [a + b for a, b in zip(n_out, n_in)]
        n = sum(sizes)
        self.n_params = n
        self.P = torch.empty(n, dtype=torch.float32, device=device)
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.g = torch.zeros(n, dtype=torch.float32, device=device)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=device)
        self.problems, self.E, self.dLdE, self.E_ref, self.loss = [], [], [], [], []
        at = 0
        for w, sz, no in zip(workloads, sizes, n_out):
            shape = (w["lens"]["n1"] + 1, w["lens"]["n2"] + 1)
            view = self.P[at:at + no].view(shape)
            view.copy_(torch.as_tensor(w["lens"]["P"], dtype=torch.float32))
            entry = None
            if sz > no:
                entry = self.P[at + no:at + sz].view(w["lens"]["n1_in"] + 1, w["lens"]["n2_in"] + 1)
                entry.copy_(torch.as_tensor(w["lens"]["P_in"], dtype=torch.float32))
            pb = api.Problem(w, ctrl_z=view, device=device, entry_z=entry)
            self.problems.append(pb)
            self.E.append(torch.zeros(pb.ext_shape, dtype=torch.float32, device=device))
            self.dLdE.append(torch.zeros(pb.ext_shape, dtype=torch.float32, device=device))
            self.E_ref.append(torch.as_tensor(w["E_ref"], dtype=torch.float32, device=device).contiguous())
            self.loss.append(torch.zeros((), dtype=torch.float64, device=device))
            at += sz
        self.grads = []
        at = 0
        for pb, sz in zip(self.problems, sizes):
            g = self.g[at:at + sz]
            self.grads.append(g.view(pb.ctrl_shape) if pb.entry_shape is None else g)
            at += sz
        self.theta = self.offset = None
        if reparam is not None:
            self._init_reparam(workloads, sizes, device)
        self.n_rays = sum(pb.n_rays for pb in self.problems)
        self.batched = len(self.problems) > 1
        # per lens: its ray order (point sources) or None
        self.orders = [pb.ray_order(self.h) if ray_order and pb.source.kind == api.FR_SOURCE_POINT else None
                       for pb in self.problems]
        self.order = None if self.batched else self.orders[0]
        if self.order is not None:
            for o in (self._fwd_opts, self._adj_opts):
                o.ray_order = self.order.data_ptr()
                o.ray_order_numel = self.order.numel()
        self.P_host = self.loss_host = None
        self.graph = None
        if graph:
            self._capture()

    def attach_host_io(self, P_host=None, loss_host=None):
        """Make every step read its control heights from host memory and write
        its losses to host memory: P_host (n_params float32, pinned) is copied
        into the device heights before the forward trace, and the loss kernels
        write loss_host (one float64 per lens, pinned; pinned host memory is
        addressable from the device) directly, in place of the device losses
        (losses() then reads loss_host). Both transfers are part of the step
        (captured into its graph), so a caller that feeds heights from the host
        and reads the loss back pays one graph launch and one synchronisation
        per step. None detaches."""
        if P_host is not None:
            if self.theta is not None:
                raise ValueError("with a reparametrisation the heights follow theta; attach no P_host")
            if (P_host.device.type != "cpu" or not P_host.is_pinned() or P_host.dtype != torch.float32
                    or P_host.numel() != self.n_params or not P_host.is_contiguous()):
                raise ValueError("P_host must be a contiguous pinned float32 CPU tensor of n_params values")
        if loss_host is not None:
            if (loss_host.device.type != "cpu" or not loss_host.is_pinned() or loss_host.dtype != torch.float64
                    or loss_host.numel() != len(self.problems) or not loss_host.is_contiguous()):
                raise ValueError("loss_host must be a contiguous pinned float64 CPU tensor, one value per lens")
        self.P_host = P_host
        self.loss_host = loss_host
        if self.graph is not None:
            self._capture()

    def _init_reparam(self, workloads, sizes, device):
        zmin, zmax = float(self.reparam["z_min"]), float(self.reparam["z_max"])
        if not zmin < zmax:
            raise ValueError("need z_min < z_max")
        off = self.reparam.get("offset")
        self.offset = torch.zeros(self.n_params, dtype=torch.float32, device=device)
        at = 0
        for k, (pb, sz) in enumerate(zip(self.problems, sizes)):
            view = self.offset[at:at + sz]
            if isinstance(off, tuple) and off[0] == "sphere":
                api.fr_offset_spherical(self.h, pb.lens, float(off[1]), float(off[2]), view)
            elif off is not None:
                arr = off[k] if isinstance(off, list) else off
                view.copy_(torch.as_tensor(np.asarray(arr), dtype=torch.float32).reshape(-1))
            at += sz
        # theta from the starting heights where they lie inside the range, else its edge
        y = (self.P - self.offset - zmin) / (0.5 * (zmax - zmin)) - 1.0
        self.theta = torch.atanh(y.clamp(-1 + 1e-6, 1 - 1e-6)).contiguous()
        if self.reparam.get("theta0") is not None:
            self.theta.copy_(torch.as_tensor(self.reparam["theta0"], dtype=torch.float32).reshape(-1))
        api.fr_reparam_tanh(self.h, self.theta, self.offset, self.n_params, zmin, zmax, self.P)

    @staticmethod
    def _accumulating(options):
        o = api.make_options() if options is None else api.Options.from_buffer_copy(options)
        o.accumulate = 1
        return o

    def _clear(self):
        # one kernel for all of them; in programmatic-launch mode 2 the forward
        # starts while it runs and waits for it before its first write
        api.fr_zero_list(self.h, list(self.E) + [self.g])

    def _forward(self):
        if self.batched:
            items = [pb.batch_item(E=E, ray_order=r) for pb, E, r in zip(self.problems, self.E, self.orders)]
            api.fr_trace_batch_forward(self.h, items, self._fwd_opts)
        else:
            pb = self.problems[0]
            api.fr_trace_forward(self.h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0, api.ALL_RAYS,
                                 self._fwd_opts, self.E[0])

    def _loss(self):
        fn = api.fr_loss_l2 if self.loss_kind == "l2" else api.fr_loss_frobenius
        for k, (pb, E, Er, d) in enumerate(zip(self.problems, self.E, self.E_ref, self.dLdE)):
            # with host I/O the loss kernel writes the pinned host buffer itself
            L = self.loss[k] if self.loss_host is None else self.loss_host.view(-1)[k:k + 1]
            fn(self.h, E, Er, pb.nx, pb.ny, pb.nu_x, pb.nu_y, L, d)

    def _adjoint(self):
        if self.batched:
            items = [pb.batch_item(dLdE=d, dLdP=g, ray_order=r)
                     for pb, d, g, r in zip(self.problems, self.dLdE, self.grads, self.orders)]
            api.fr_trace_batch_adjoint(self.h, items, self._adj_opts)
        else:
            pb = self.problems[0]
            api.fr_trace_adjoint(self.h, pb.lens, pb.source, pb.target, pb.n_rays, pb.seed, 0, api.ALL_RAYS,
                                 self._adj_opts, self.dLdE[0], self.grads[0])

    def _adam(self):
        if self.theta is None:
            api.fr_adam_step(self.h, self.P, self.m, self.v, self.g, self.n_params, self.lr, self.betas[0],
                             self.betas[1], self.eps, self.step_count)
        else:
            api.fr_adam_step_tanh(self.h, self.theta, self.m, self.v, self.g, self.offset, self.n_params, self.lr,
                                  self.betas[0], self.betas[1], self.eps, float(self.reparam["z_min"]),
                                  float(self.reparam["z_max"]), self.step_count, self.P)

    def eager_step(self):
        if self.P_host is not None:
            self.P.copy_(self.P_host, non_blocking=True)
        self._clear()
        # mode 2: the forward follows the clearing kernel and the adjoint the
        # loss kernel, neither of which writes the lens
        api.fr_set_programmatic_launch(self.h, 2 if self.pdl else 0)
        try:
            self._forward()
            self._loss()
            self._adjoint()
            self._adam()
        finally:
            api.fr_set_programmatic_launch(self.h, 0)

    def _capture(self):
        state = self._state()
        saved = [t.clone() for t in state]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.eager_step()          # sizes the handle's scratch memory before capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.eager_step()
        torch.cuda.synchronize()
        for t, v in zip(state, saved):
            t.copy_(v)
        torch.cuda.synchronize()

    def _state(self):
        st = [self.P, self.m, self.v, self.step_count]
        return st + ([self.theta] if self.theta is not None else [])

    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.eager_step()

    def losses(self):
        if self.loss_host is not None:
            torch.cuda.synchronize()
            return self.loss_host.view(-1).clone()
        return torch.stack(self.loss).cpu()

    # Checkpoint and resume: the optimiser's whole state. Rays are functions of
    # (seed, id), so a resumed run continues exactly (bit for bit in
    # deterministic mode).
    def state_dict(self):
        st = {"P": self.P.clone(), "m": self.m.clone(), "v": self.v.clone(), "step": self.step_count.clone(),
              "lr": self.lr, "betas": self.betas, "eps": self.eps, "loss": self.loss_kind,
              "seeds": [pb.seed for pb in self.problems], "n_rays": [pb.n_rays for pb in self.problems]}
        if self.theta is not None:
            st["theta"] = self.theta.clone()
            st["offset"] = self.offset.clone()
            st["reparam"] = {k: v for k, v in self.reparam.items() if k in ("z_min", "z_max")}
        return st

    def load_state_dict(self, st):
        if st["seeds"] != [pb.seed for pb in self.problems] or st["n_rays"] != [pb.n_rays for pb in self.problems]:
            raise ValueError("the checkpoint is of other rays")
        if (st.get("theta") is None) != (self.theta is None) or st["P"].numel() != self.P.numel():
            raise ValueError("the checkpoint is of another parametrisation")
        torch.cuda.synchronize()
        for name in ("P", "m", "v"):
            getattr(self, name).copy_(st[name])
        self.step_count.copy_(st["step"])
        if self.theta is not None:
            self.theta.copy_(st["theta"])
            self.offset.copy_(st["offset"])
        torch.cuda.synchronize()

    def save(self, path):
        torch.save(self.state_dict(), path)

    def load(self, path):
        self.load_state_dict(torch.load(path, map_location=self.P.device, weights_only=False))

    # Kernel launches per step (for the launch count of a timed region).
    def launches_per_step(self):
        n_items = len(self.problems)
        det = bool(self.options is not None and self.options.deterministic)
        mesh = bool(self.options is not None and self.options.mesh_nu > 0)
        # point sources with a flat entry face, intersected by Newton: a deferred pass after each trace
        deferred = int(not mesh and any(pb.source.kind == api.FR_SOURCE_POINT and pb.entry_shape is None
                                        for pb in self.problems))
        fwd = 1 + deferred + (n_items if det else 0)      # trace (+ deferred pass) (+ fixed->float)
        adj = 1 + deferred + (2 * n_items if det else 0)  # trace (+ deferred pass) (+ absmax, fixed->float)
        return 1 + fwd + n_items + adj + 1                # clearing kernel + ... + one loss per lens + Adam
