"""The whole hot path (Steps II-IV) captured once into a CUDA graph and replayed
(PipelineGraph); matrices streamed from pinned host memory with overlapped uploads
(StreamingPipeline); many learn problems in one graph (BatchedLearnGraph).

Every buffer is allocated up front; capture records the asynchronous entry points
(dopinf_transform, dopinf_gram_async, dopinf_reduce_async, dopinf_learn_async), which neither
synchronise nor copy from the host, so a replay reruns the transform, the Gram, the eigensolve
and projection, the regularised solves, the rollouts and the selection with one launch from
the host.  Failures (a kernel timeout, a rank failure, no valid candidate) are OR-ed into one
device flag word that the caller reads when it wants to.
"""
import ctypes

import torch

from . import dopinf as dp


class PipelineGraph:
    def __init__(self, Q, var_row_offsets, r_cap, r_list, beta1, beta2, n_steps, mode=dp.DISCRETE, dt=1.0,
                 gram_mode=dp.GRAM_OZAKI_FP64, r_fixed=None, energy_target=0.9996, max_growth=1.2, share=None,
                 share_back=None):
        """share: another PipelineGraph of the same sizes whose workspaces and output buffers
        this one reuses (both graphs then run on one stream, one after the other).
        share_back: another PipelineGraph whose reduce and learn workspaces and outputs this one
        reuses, with transform and Gram buffers (mean, scale, D, flags, their workspaces) of its
        own: the front of one may then run beside the back of the other, the backs in turn."""
        self.Q = Q
        n, k, ldq = dp._colmajor(Q)
        dev = Q.device
        self.n, self.k, self.ldq = n, k, ldq
        self.offs = (dp._c_i64 * len(var_row_offsets))(*[int(v) for v in var_row_offsets])
        self.n_vars = len(var_row_offsets) - 1
        self.r_cap = int(r_cap)
        self.r_fixed = int(r_cap if r_fixed is None else r_fixed)
        self.energy_target = float(energy_target)
        self.gram_mode = gram_mode
        self.r_list = [int(r) for r in r_list]
        self.beta1 = [float(b) for b in beta1]
        self.beta2 = [float(b) for b in beta2]
        self.n_steps, self.mode, self.dt, self.max_growth = int(n_steps), int(mode), float(dt), float(max_growth)
        f64, i32 = torch.float64, torch.int32
        self.graph = None
        if share is not None:
            if (share.n, share.k, share.r_cap, share.r_list, share.gram_mode) != (n, k, self.r_cap, self.r_list,
                                                                                 gram_mode):
                raise ValueError("share: the pipelines differ in size")
            for name in ("flags", "mean", "scale", "D", "red", "res", "ws", "wbuf", "wsz"):
                setattr(self, name, getattr(share, name))
            return
        if share_back is not None:
            if (share_back.k, share_back.r_cap, share_back.r_list) != (k, self.r_cap, self.r_list):
                raise ValueError("share_back: the pipelines differ in size")
        self.flags = torch.zeros(1, dtype=i32, device=dev)
        self.mean = torch.empty(n, dtype=f64, device=dev)
        self.scale = torch.empty(self.n_vars, dtype=f64, device=dev)
        self.D = torch.zeros(k, k, dtype=f64, device=dev)
        if share_back is not None:
            self.red, self.res = share_back.red, share_back.res
            sizes = [dp.lib.dopinf_transform_workspace(n, self.n_vars),
                     dp.lib.dopinf_gram_workspace(n, k, dp._dtype_code(Q), gram_mode)]
            self.ws = [dp.Workspace(dev) for _ in sizes] + share_back.ws[2:]
            self.wbuf = [w.get(nb) for w, nb in zip(self.ws, sizes)] + share_back.wbuf[2:]
            self.wsz = sizes + share_back.wsz[2:]
            return
        self.red = dict(eigvals=torch.empty(r_cap, dtype=f64, device=dev),
                        Tr=torch.empty(r_cap, k, dtype=f64, device=dev).t(),
                        Qhat=torch.empty(k, r_cap, dtype=f64, device=dev).t(),
                        r=torch.zeros(1, dtype=i32, device=dev), trace=torch.zeros(1, dtype=f64, device=dev))
        n_cand = len(self.r_list) * len(self.beta1) * len(self.beta2)
        d_max = max(r + r * (r + 1) // 2 + 1 for r in self.r_list)
        self.res = dict(train_err=torch.empty(n_cand, dtype=f64, device=dev),
                        growth=torch.empty(n_cand, dtype=f64, device=dev),
                        status=torch.empty(n_cand, dtype=i32, device=dev),
                        steps=torch.zeros(n_cand, dtype=torch.int64, device=dev),
                        best=torch.zeros(1, dtype=i32, device=dev),
                        O_best=torch.zeros(d_max, r_cap, dtype=f64, device=dev).t())
        # one workspace per stage, sized before capture
        rl = (ctypes.c_int * len(self.r_list))(*self.r_list)
        sizes = [dp.lib.dopinf_transform_workspace(n, self.n_vars),
                 dp.lib.dopinf_gram_workspace(n, k, dp._dtype_code(Q), gram_mode),
                 dp.lib.dopinf_reduce_workspace(k, r_cap),
                 dp.lib.dopinf_learn_workspace(r_cap, k, rl, len(self.r_list), len(self.beta1), len(self.beta2))]
        self.ws = [dp.Workspace(dev) for _ in sizes]
        self.wbuf = [w.get(nb) for w, nb in zip(self.ws, sizes)]
        self.wsz = sizes

    def _launch(self, stream, front=True, back=True, learn=True):
        """The pipeline on `stream` through the asynchronous entry points (no host synchronisation):
        front = transform and Gram (the steps that read Q), back = reduce, then learn (unless
        learn is False)."""
        L, P, s = dp.lib, dp._ptr, dp._stream(stream)
        red, res = self.red, self.res
        if front:
            dp._check("dopinf_transform", L.dopinf_transform(
                P(self.Q), dp._dtype_code(self.Q), self.n, self.k, self.ldq, self.n_vars, self.offs,
                dp.CENTER | dp.SCALE, P(self.mean), P(self.scale), P(self.flags), P(self.wbuf[0]), self.wsz[0],
                s))
            dp._check("dopinf_gram_async", L.dopinf_gram_async(
                P(self.Q), dp._dtype_code(self.Q), self.n, self.k, self.ldq, self.gram_mode, 0, P(self.D),
                self.D.stride(0), P(self.flags), P(self.wbuf[1]), self.wsz[1], s))
        if not back:
            return
        dp._check("dopinf_reduce_async", L.dopinf_reduce_async(
            P(self.D), self.k, self.D.stride(0), self.energy_target, self.r_fixed, self.r_cap, P(red["r"]),
            P(red["trace"]), P(red["eigvals"]), P(red["Tr"]), P(red["Qhat"]), P(self.flags), P(self.wbuf[2]),
            self.wsz[2], s))
        if not learn:
            return
        self._launch_learn(stream)

    def _launch_learn(self, stream):
        L, P, s = dp.lib, dp._ptr, dp._stream(stream)
        red, res = self.red, self.res
        rl = (ctypes.c_int * len(self.r_list))(*self.r_list)
        b1 = (ctypes.c_double * len(self.beta1))(*self.beta1)
        b2 = (ctypes.c_double * len(self.beta2))(*self.beta2)
        Qh = red["Qhat"]
        dp._check("dopinf_learn_async", L.dopinf_learn_async(
            P(Qh), self.r_cap, self.k, Qh.stride(1), rl, len(self.r_list), b1, len(self.beta1), b2,
            len(self.beta2), self.mode, self.dt, self.n_steps, self.max_growth, P(res["train_err"]),
            P(res["growth"]), P(res["status"]), P(res["steps"]), P(res["best"]), P(res["O_best"]),
            P(self.flags), P(self.wbuf[3]), self.wsz[3], s))

    def run_eager(self, stream=None):
        """One pass without the graph (the same launches, issued from the host)."""
        self._launch(stream if stream is not None else torch.cuda.current_stream())

    def capture(self, split=False):
        """Capture the pipeline into a CUDA graph (after one eager warm-up pass).  split: two
        graphs instead, graph_front (transform, Gram) and graph_back (reduce, learn), replayed by
        replay_front / replay_back, so that a caller may place work between them; split = 3:
        graph_back is the reduce alone and graph_learn the learn step (replay_learn)."""
        side = torch.cuda.Stream(device=self.Q.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._launch(side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        if split:
            self.graph_front, self.graph_back = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph_front):
                self._launch(torch.cuda.current_stream(), back=False)
            with torch.cuda.graph(self.graph_back):
                self._launch(torch.cuda.current_stream(), front=False, learn=split != 3)
            if split == 3:
                self.graph_learn = torch.cuda.CUDAGraph()
                with torch.cuda.graph(self.graph_learn):
                    self._launch_learn(torch.cuda.current_stream())
            return self
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._launch(torch.cuda.current_stream())
        return self

    def replay(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self.graph_front.replay()
            self.graph_back.replay()

    def replay_front(self):
        self.graph_front.replay()

    def replay_back(self):
        self.graph_back.replay()

    def replay_learn(self):
        self.graph_learn.replay()

    def flags_value(self):
        """The OR of the DOPINF_FLAG_* bits raised so far (synchronises)."""
        return int(self.flags.item())


def bind_host_to_device(device):
    """Restrict this process to the CPUs attached to `device` (sysfs local_cpulist of its PCI
    function), so that host buffers allocated afterwards (first touch) sit on the memory node
    nearest to it and its host-device copies take the shortest path.  Returns the CPU list, or
    None where the topology is not published (nothing is changed then)."""
    import os
    try:
        p = torch.cuda.get_device_properties(torch.device(device))
        bus = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        with open("/sys/bus/pci/devices/%s/local_cpulist" % bus) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except (OSError, ValueError, AttributeError, RuntimeError):
        return None


def upload(dst, src, chunks=8):
    """Host-to-device copy of a (k, n) snapshot block as `chunks` copies of consecutive
    snapshots on the current stream (one copy engine request per chunk instead of one for the
    whole matrix)."""
    rows = dst.shape[0]
    for c in range(chunks):
        a, b = rows * c // chunks, rows * (c + 1) // chunks
        if b > a:
            dst[a:b].copy_(src[a:b], non_blocking=True)


class OverlappedPipeline:
    """Consecutive pipelines over two device-resident snapshot matrices (step i on copy i mod 2),
    each step's front (transform, Gram: tensor cores and HBM) on a front stream beside the
    previous step's learn step (rollouts: the FP64 pipe, most SMs idle in their tail) on the
    compute stream.  The reduce steps stay in turn on the compute stream and no front runs beside
    them (the tridiagonalisation is a cooperative launch whose CTAs must all be resident), and
    the learn steps share one set of buffers, so they run one after the other.

        front(i)  after reduce(i - 1)           (front stream)
        reduce(i) after front(i) and learn(i-1) (compute stream)
        learn(i)  after reduce(i)               (compute stream)

    Every step computes its full pipeline; a step's results (res, red, flags of its copy) stay
    valid until the next step's reduce starts."""

    def __init__(self, Qs, var_row_offsets, r_cap, r_list, beta1, beta2, n_steps, mode=dp.DISCRETE, dt=1.0,
                 gram_mode=dp.GRAM_OZAKI_FP64, r_fixed=None, energy_target=0.9996, max_growth=1.2):
        """Qs: two column-major (n x k) device matrices of the same shape, the snapshot matrix of
        even and odd steps (each is transformed in place by its steps)."""
        if len(Qs) != 2:
            raise ValueError("Qs: two snapshot matrices")
        kw = dict(mode=mode, dt=dt, gram_mode=gram_mode, r_fixed=r_fixed, energy_target=energy_target,
                  max_growth=max_growth)
        dev = Qs[0].device
        self.pg = [PipelineGraph(Qs[0], var_row_offsets, r_cap, r_list, beta1, beta2, n_steps, **kw)]
        self.pg.append(PipelineGraph(Qs[1], var_row_offsets, r_cap, r_list, beta1, beta2, n_steps,
                                     share_back=self.pg[0], **kw))
        for pg in self.pg:
            pg.capture(split=3)
        torch.cuda.synchronize(dev)
        self.front_stream = torch.cuda.Stream(device=dev)
        self.stream = torch.cuda.Stream(device=dev)
        self.gram_done = [torch.cuda.Event() for _ in range(2)]
        self.reduce_done = torch.cuda.Event()
        self.reduce_done.record(torch.cuda.current_stream(dev))
        self.count = 0

    def submit(self, refill=None):
        """Queue the next step; returns its index (its copy is index mod 2).  refill(Q): called
        on the front stream before the step's transform, to enqueue writes of the step's input
        into its copy Q (a device copy, an upload)."""
        i, b = self.count, self.count % 2
        pg = self.pg[b]
        self.front_stream.wait_event(self.reduce_done)
        with torch.cuda.stream(self.front_stream):
            if refill is not None:
                refill(pg.Q)
            pg.replay_front()
            self.gram_done[b].record(self.front_stream)
        self.stream.wait_event(self.gram_done[b])
        with torch.cuda.stream(self.stream):
            pg.replay_back()
            self.reduce_done.record(self.stream)
            pg.replay_learn()
        self.count += 1
        return i

    def join(self, stream=None):
        """Make `stream` (default: the current stream) wait for everything submitted."""
        st = stream if stream is not None else torch.cuda.current_stream()
        st.wait_stream(self.front_stream)
        st.wait_stream(self.stream)

    def start_after(self, stream=None):
        """Make the next submitted step wait for the work queued so far on `stream`."""
        st = stream if stream is not None else torch.cuda.current_stream()
        self.front_stream.wait_stream(st)
        self.stream.wait_stream(st)

    def results(self, i):
        """Step i's outputs (device tensors; synchronises on the compute stream): valid for the
        latest submitted step until another is submitted."""
        if i != self.count - 1:
            raise ValueError("only the latest step's results are held")
        self.stream.synchronize()
        pg = self.pg[i % 2]
        return dict(res=pg.res, red=pg.red, flags=int(pg.flags.item()))


class StreamingPipeline:
    """Steps II-IV over snapshot matrices that arrive one after another in pinned host memory.

    Two device copies of the snapshot matrix, each with its own captured front graph
    (transform and Gram, the steps that read the matrix) and buffers; reduce and learn share
    their workspaces and outputs.  Three streams, the schedule of OverlappedPipeline plus the
    uploads: the upload of a matrix into a copy (copy stream) waits only for the front that last
    read that copy (two steps back); a step's front (front stream) waits for its upload and for
    the previous step's reduce, and so runs beside the previous step's learn step; reduce and
    learn run in turn on the compute stream.  Each step's results (training errors, statuses,
    the best index and its operators, the failure flags) are copied back into pinned host memory
    on the compute stream; result(i) waits for step i's copy and returns them.
    """

    OUTS = ("train_err", "status", "best", "O_best")

    def __init__(self, host_QT, var_row_offsets, r_cap, r_list, beta1, beta2, n_steps, mode=dp.DISCRETE,
                 dt=1.0, gram_mode=dp.GRAM_OZAKI_FP64, r_fixed=None, energy_target=0.9996, max_growth=1.2,
                 device="cuda", upload_chunks=8, record_times=False):
        """host_QT: pinned CPU tensor (k, n), row-major, i.e. the column-major n x k snapshot matrix;
        every submitted matrix has this shape and dtype.  The first one also serves for capture.
        record_times: bracket every upload and every step's compute with timing events
        (step_times(i) reads them), to see whether the uploads hide behind the compute."""
        if not host_QT.is_pinned():
            raise ValueError("host_QT must be in pinned host memory")
        dev = torch.device(device)
        self.upload_chunks = int(upload_chunks)
        self.QT = [torch.empty(host_QT.shape, dtype=host_QT.dtype, device=dev) for _ in range(2)]
        kw = dict(mode=mode, dt=dt, gram_mode=gram_mode, r_fixed=r_fixed, energy_target=energy_target,
                  max_growth=max_growth)
        self.pg = []
        for b in range(2):
            self.QT[b].copy_(host_QT)
            share_back = self.pg[0] if b else None
            self.pg.append(PipelineGraph(self.QT[b].t(), var_row_offsets, r_cap, r_list, beta1, beta2, n_steps,
                                         share_back=share_back, **kw).capture(split=3))
        torch.cuda.synchronize(dev)
        self.stream = torch.cuda.Stream(device=dev)
        self.front_stream = torch.cuda.Stream(device=dev)
        self.copy_stream = torch.cuda.Stream(device=dev)
        self.front_done = [torch.cuda.Event() for _ in range(2)]  # the last front graph on QT[b] finished
        self.uploaded = [torch.cuda.Event() for _ in range(2)]    # QT[b] holds the next matrix
        self.fetched = [torch.cuda.Event() for _ in range(2)]     # host slot b holds a step's results
        self.reduce_done = torch.cuda.Event()                     # the last reduce finished
        for e in self.front_done:
            e.record(torch.cuda.current_stream(dev))
        self.reduce_done.record(torch.cuda.current_stream(dev))
        pg = self.pg[0]
        srcs = [pg.res[name] for name in self.OUTS] + [pg.flags]
        self.host_out = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in srcs] for _ in range(2)]
        self.h2d_bytes = host_QT.numel() * host_QT.element_size()
        self.d2h_bytes = sum(t.numel() * t.element_size() for t in srcs)
        self.count = 0
        self.times = {} if record_times else None

    def submit(self, host_QT):
        """Queue one step on host_QT (pinned, the shape of the first); returns its index.

        The upload from host_QT is asynchronous and may still be running when this returns:
        the caller must not refill or free host_QT until upload_event(i) has completed (or
        result(i) has returned); rotate several pinned buffers to keep filling meanwhile."""
        i, b = self.count, self.count % 2
        pg = self.pg[b]
        # the upload into copy b waits for the front graph that last read it (step i - 2)
        tm = None
        if self.times is not None:
            tm = self.times[i] = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        self.copy_stream.wait_event(self.front_done[b])
        with torch.cuda.stream(self.copy_stream):
            if tm:
                tm[0].record(self.copy_stream)
            upload(self.QT[b], host_QT, self.upload_chunks)
            if tm:
                tm[1].record(self.copy_stream)
            self.uploaded[b].record(self.copy_stream)
        self.front_stream.wait_event(self.uploaded[b])
        self.front_stream.wait_event(self.reduce_done)
        with torch.cuda.stream(self.front_stream):
            if tm:
                tm[2].record(self.front_stream)
            pg.replay_front()
            self.front_done[b].record(self.front_stream)
        self.stream.wait_event(self.front_done[b])
        with torch.cuda.stream(self.stream):
            pg.replay_back()
            self.reduce_done.record(self.stream)
            if tm:
                tm[4].record(self.stream)
            pg.replay_learn()
            if tm:
                tm[3].record(self.stream)
            srcs = [pg.res[name] for name in self.OUTS] + [pg.flags]
            for dst, src in zip(self.host_out[b], srcs):
                dst.copy_(src, non_blocking=True)
            pg.flags.zero_()
            self.fetched[b].record(self.stream)
        self.count += 1
        return i

    def upload_event(self, i):
        """CUDA event recorded when step i's upload has finished (valid until step i + 2 is
        submitted): host_QT of step i may be reused once it has completed."""
        if not (self.count - 2 <= i < self.count):
            raise ValueError("step %d is no longer (or not yet) held" % i)
        return self.uploaded[i % 2]

    def step_times(self, i):
        """(upload ms, span ms, upload wait ms) of step i (waits for it; record_times=True): the
        span runs from the start of the step's transform to the end of its learn step; the wait
        is how long the step's upload ended after the previous step's reduce, i.e. how long the
        front waited for its input (None for step 0)."""
        if self.times is None:
            raise ValueError("constructed without record_times")
        tm = self.times[i]
        tm[3].synchronize()
        wait = None
        if i - 1 in self.times:
            wait = max(0.0, self.times[i - 1][4].elapsed_time(tm[1]))
        return tm[0].elapsed_time(tm[1]), tm[2].elapsed_time(tm[3]), wait

    def result(self, i):
        """Step i's results on the host (waits for them); valid until step i + 2 is submitted."""
        if not (self.count - 2 <= i < self.count):
            raise ValueError("result %d is no longer (or not yet) held" % i)
        b = i % 2
        self.fetched[b].synchronize()
        out = dict(zip(self.OUTS, (t.clone() for t in self.host_out[b][:-1])))
        out["best"] = int(out["best"][0])
        out["flags"] = int(self.host_out[b][-1][0])
        return out

    def run(self, host_mats):
        """Every matrix of host_mats through the pipeline; returns the list of results."""
        out, first = [], self.count
        for m in host_mats:
            i = self.submit(m)
            if i > first:
                out.append(self.result(i - 1))
        if self.count > first:
            out.append(self.result(self.count - 1))
        return out


class BatchedLearnGraph:
    """Many independent learn problems (each its own reduced data Qhat, r list and grid) captured
    into one CUDA graph: problem p runs on its own capture stream, forked from and joined back
    to the capturing stream, so the graph's branches run concurrently.  Buffers per problem
    are allocated up front; results stay on the device."""

    def __init__(self, problems, n_steps, mode=dp.DISCRETE, dt=1.0, max_growth=1.2):
        """problems: list of dict(Qhat=(r_max, k) column-major device tensor, r_list=[...],
        beta1=[...], beta2=[...])."""
        self.problems = problems
        self.n_steps, self.mode, self.dt, self.max_growth = int(n_steps), int(mode), float(dt), float(max_growth)
        self.out = []
        self.bufs = []
        for pr in problems:
            Qh = pr["Qhat"]
            r_max, k = Qh.shape
            dev = Qh.device
            n_cand = len(pr["r_list"]) * len(pr["beta1"]) * len(pr["beta2"])
            d_max = max(r + r * (r + 1) // 2 + 1 for r in pr["r_list"])
            self.out.append(dict(train_err=torch.empty(n_cand, dtype=torch.float64, device=dev),
                                 growth=torch.empty(n_cand, dtype=torch.float64, device=dev),
                                 status=torch.empty(n_cand, dtype=torch.int32, device=dev),
                                 steps=torch.zeros(n_cand, dtype=torch.int64, device=dev),
                                 best=torch.zeros(1, dtype=torch.int32, device=dev),
                                 O_best=torch.zeros(d_max, r_max, dtype=torch.float64, device=dev).t(),
                                 flags=torch.zeros(1, dtype=torch.int32, device=dev)))
            rl = (ctypes.c_int * len(pr["r_list"]))(*[int(r) for r in pr["r_list"]])
            nb = dp.lib.dopinf_learn_workspace(r_max, k, rl, len(pr["r_list"]), len(pr["beta1"]), len(pr["beta2"]))
            w = dp.Workspace(dev)
            self.bufs.append(w)
            w.get(nb)
        self.streams = [torch.cuda.Stream(device=problems[0]["Qhat"].device) for _ in problems]
        self.graph = None

    def _launch(self):
        main = torch.cuda.current_stream()
        for s in self.streams:
            s.wait_stream(main)
        for pr, out, w, s in zip(self.problems, self.out, self.bufs, self.streams):
            with torch.cuda.stream(s):
                dp.dopinf_learn_async(pr["Qhat"], pr["r_list"], pr["beta1"], pr["beta2"], self.n_steps, out,
                                      mode=self.mode, dt=self.dt, max_growth=self.max_growth, ws=w, stream=s)
        for s in self.streams:
            main.wait_stream(s)

    def capture(self):
        self._launch()  # eager warm-up
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._launch()
        return self

    def replay(self):
        self.graph.replay()
