"""The edge batch of one planning iteration, run through the C ABI:
parents (fn_knn_tree) -> edges (fn_make_edges) -> goal edges at their fixed
duration and free edges by the capped duration scan (fn_time_edges)."""
from __future__ import annotations

import numpy as np
import torch

from . import ops


class EdgeBatchRunner:
    def __init__(self, w, k, S, device, stream=None):
        self.w, self.k, self.S, self.dev = w, k, S, device
        self.arm = w["arm"]
        self.grid = np.asarray(w["grid"], np.float32)
        self.n_goal = w["goal"].shape[0]
        cand = np.concatenate([w["goal"], w["free"]])
        self.B = cand.shape[0]
        self.E = self.B * k
        self.Eg = self.n_goal * k
        self.h_tree = torch.from_numpy(w["tree"]).pin_memory()
        self.h_t = torch.from_numpy(w["t_node"]).pin_memory()
        self.h_cand = torch.from_numpy(cand).pin_memory()
        self.h_treq = torch.from_numpy(w["t_req"]).pin_memory()
        self.tree = self.h_tree.to(device)
        self.t_node = self.h_t.to(device)
        self.cand = self.h_cand.to(device)
        self.t_req = self.h_treq.to(device)
        self.t_best = float(w["t_best"])
        N = self.tree.shape[0]
        need = ops.knn_workspace_bytes(self.B, N, k - 1)
        self.ws = torch.empty(need + 256, dtype=torch.uint8, device=device)
        self.nn = (torch.empty(self.B, k - 1, dtype=torch.int32, device=device),
                   torch.empty(self.B, k - 1, dtype=torch.float32, device=device))
        self.edges = (torch.empty(self.E, 16, device=device), torch.empty(self.E, 16, device=device),
                      torch.empty(self.E, device=device),
                      torch.empty(self.E, dtype=torch.int32, device=device))
        self.res_g = self._out(self.Eg)
        self.res_f = self._out(self.E - self.Eg)
        self.edges_per_step = self.E
        self.launches_per_step = (2 if need > 0 else 1) + 1 + 2

    def _out(self, n):
        d = self.dev
        return dict(k_star=torch.empty(n, dtype=torch.int32, device=d),
                    T_star=torch.empty(n, device=d), rho3=torch.empty(n, 3, device=d),
                    ok=torch.empty(n, dtype=torch.uint8, device=d))

    def step(self, kernel_events=None, counter=None):
        ops.knn_tree(self.tree, self.cand, self.k - 1, 0.1, first=1, workspace=self.ws, out=self.nn)
        s0, s1, Tp, _ = ops.make_edges(self.tree, self.t_node, self.cand, self.n_goal, self.nn[0],
                                       self.t_req, self.t_best, out=self.edges)
        Eg = self.Eg
        ops.time_edges(self.arm, s0[:Eg], s1[:Eg], None, self.S, mode=ops.FN_MODE_FIXED,
                       T_fixed=Tp[:Eg], out=self.res_g,
                       sample_count=None if counter is None else counter[0:1])
        if kernel_events:
            kernel_events[0].record()
        ops.time_edges(self.arm, s0[Eg:], s1[Eg:], self.grid, self.S, T_cap=Tp[Eg:],
                       out=self.res_f, sample_count=None if counter is None else counter[1:2])
        if kernel_events:
            kernel_events[1].record()

    def count_samples(self):
        c = torch.zeros(2, dtype=torch.int64, device=self.dev)
        self.step(counter=c)
        torch.cuda.synchronize()
        c = c.cpu().numpy()
        return {"goal": int(c[0]), "free": int(c[1])}

    def results(self):
        self.step()
        torch.cuda.synchronize()
        return self.res_f["k_star"].cpu().numpy(), self.res_g["k_star"].cpu().numpy()

    def e2e(self, steps):
        """Same step with the inputs copied from pinned host memory and the
        per-edge results copied back, timed with events on the stream."""
        st = torch.cuda.current_stream()
        outs = [torch.empty(self.E, dtype=torch.int32).pin_memory(),
                torch.empty(self.E, dtype=torch.float32).pin_memory(),
                torch.empty(self.E, dtype=torch.uint8).pin_memory()]
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(steps):
            self.tree.copy_(self.h_tree, non_blocking=True)
            self.t_node.copy_(self.h_t, non_blocking=True)
            self.cand.copy_(self.h_cand, non_blocking=True)
            self.t_req.copy_(self.h_treq, non_blocking=True)
            self.step()
            Eg = self.Eg
            outs[0][:Eg].copy_(self.res_g["k_star"], non_blocking=True)
            outs[0][Eg:].copy_(self.res_f["k_star"], non_blocking=True)
            outs[1][:Eg].copy_(self.res_g["T_star"], non_blocking=True)
            outs[1][Eg:].copy_(self.res_f["T_star"], non_blocking=True)
            outs[2][:Eg].copy_(self.res_g["ok"], non_blocking=True)
            outs[2][Eg:].copy_(self.res_f["ok"], non_blocking=True)
        b.record(st)
        b.synchronize()
        h2d = (self.h_tree.numel() + self.h_t.numel() + self.h_cand.numel() + self.h_treq.numel()) * 4
        d2h = self.E * (4 + 4 + 1)
        return a.elapsed_time(b) / steps, h2d, d2h
