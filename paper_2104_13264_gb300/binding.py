"""ctypes binding of libtnmc.so (argument marshalling only).

Every computation happens in the CUDA library; this module passes pointers
and sizes.  Device memory comes from torch tensors; calls are enqueued on the
current torch CUDA stream unless one is given.  If the library is missing,
``lib()`` raises: there is no fallback path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtnmc.so")

F64, F32, BF16 = 0, 1, 2
PRECISIONS = {"f64": F64, "f32": F32, "bf16": BF16}
FLAG_NUMERIC = 1

_lib = None


class TnmcError(RuntimeError):
    pass


class _Lattice(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("Jh", ctypes.c_void_p),
                ("Jv", ctypes.c_void_p), ("h", ctypes.c_void_p)]


class _Info(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("chi", ctypes.c_int), ("pad", ctypes.c_int),
                ("precision_mask", ctypes.c_int), ("integer_couplings", ctypes.c_int),
                ("beta", ctypes.c_double), ("logZ", ctypes.c_double), ("bytes", ctypes.c_int64)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("precision", ctypes.c_int), ("tile", ctypes.c_int), ("order", ctypes.c_int),
                ("grid", ctypes.c_int), ("chains", ctypes.c_int64), ("proposal_rows", ctypes.c_int64),
                ("proposal_bytes", ctypes.c_int64), ("chain_rows", ctypes.c_int64), ("chain_bytes", ctypes.c_int64),
                ("items", ctypes.c_int64), ("smem_bytes", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_INT = ctypes.c_int

SIGNATURES = {
    "tnmc_last_error": ([], ctypes.c_char_p),
    "tnmc_build_env": ([ctypes.POINTER(_Lattice), ctypes.c_double, _INT, _INT, _P, ctypes.POINTER(_P)], _INT),
    "tnmc_build_env_bond": ([ctypes.POINTER(_Lattice), ctypes.c_double, _INT, _INT, _P, ctypes.POINTER(_P)], _INT),
    "tnmc_build_env_variational": ([ctypes.POINTER(_Lattice), ctypes.c_double, _INT, _INT, _INT, _P,
                                    ctypes.POINTER(_P)], _INT),
    "tnmc_env_free": ([_P], _INT),
    "tnmc_env_set_order": ([_P, _INT], _INT),
    "tnmc_env_info": ([_P, ctypes.POINTER(_Info)], _INT),
    "tnmc_env_export": ([_P, _P, _P, _P, _P, _P], _INT),
    "tnmc_env_status": ([_P, ctypes.POINTER(ctypes.c_int32)], _INT),
    "tnmc_sample": ([_P, _INT, _I64, _U64, _U64, _P, _P, _P, _P, _P], _INT),
    "tnmc_logq": ([_P, _INT, _I64, _P, _P, _P, _P, _P], _INT),
    "tnmc_sample_noalloc": ([_P, _INT, _I64, _U64, _U64, _P, _P, _P, _P, _P], _INT),
    "tnmc_init_chains": ([_P, _INT, _I64, _U64, _P, _P, _P, _P], _INT),
    "tnmc_mh_step": ([_P, _I64, _I64, _P, _P, _P, _P, _P, _P, _U64, _U64, _P, _P, _P], _INT),
    "tnmc_logq_backward": ([_P, _I64, _P, _P, _P, _P], _INT),
    "tnmc_env_get_params": ([_P, _P, _P], _INT),
    "tnmc_env_set_params": ([_P, _P, _P], _INT),
    "tnmc_env_set_tensors": ([_P, _P, _P], _INT),
    "tnmc_build_env_batched": ([_INT, _P, _P, _P, _INT, _P, _P], _INT),
    "tnmc_batch_create": ([_INT, _P, _P, _I64, _INT, _INT, _INT, _P, ctypes.POINTER(_P)], _INT),
    "tnmc_batch_free": ([_P], _INT),
    "tnmc_batch_info": ([_P, ctypes.POINTER(_BatchInfo)], _INT),
    "tnmc_batch_layout": ([_P, _P, _P, _P, _P], _INT),
    "tnmc_batch_set_step": ([_P, _U64, _U64, _P], _INT),
    "tnmc_batch_balance": ([_P, _P, _P], _INT),
    "tnmc_batch_advance": ([_P, _P], _INT),
    "tnmc_sample_batched": ([_P, _P, _P, _P, _P, _P], _INT),
    "tnmc_logq_batched": ([_P, _P, _P, _P, _P, _P], _INT),
    "tnmc_batch_init_chains": ([_P, _U64, _P, _P, _P, _P], _INT),
    "tnmc_mh_batched": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P], _INT),
    "tnmc_set_allocator": ([_P, _P, _P], _INT),
    "tnmc_metropolis": ([_P, _INT, _I64, _P, _P, _P, _U64, _U64, _U64, _INT, _P], _INT),
    "tnmc_link_overlap": ([_P, _I64, _P, _P, _P], _INT),
    "tnmc_metropolis_batched": ([_P, _P, _P, _P, _INT, _P], _INT),
    "tnmc_link_overlap_batched": ([_P, _P, _P, _P], _INT),
}

class _Lattice3D(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("Lz", ctypes.c_int), ("Jx", ctypes.c_void_p),
                ("Jy", ctypes.c_void_p), ("Jz", ctypes.c_void_p), ("h", ctypes.c_void_p)]


SIGNATURES.update({
    "tnmc3d_build_env": ([ctypes.POINTER(_Lattice3D), ctypes.c_double, _INT, _INT, _P, ctypes.POINTER(_P)], _INT),
    "tnmc3d_build_env_bond": ([ctypes.POINTER(_Lattice3D), ctypes.c_double, _INT, _INT, _P, ctypes.POINTER(_P)],
                              _INT),
    "tnmc3d_env_free": ([_P], _INT),
    "tnmc3d_env_status": ([_P, ctypes.POINTER(ctypes.c_int32)], _INT),
    "tnmc3d_env_export": ([_P, _P, _P, _P], _INT),
    "tnmc3d_sample": ([_P, _INT, _I64, _U64, _U64, _P, _P, _P, _P, _P], _INT),
    "tnmc3d_logq": ([_P, _INT, _I64, _P, _P, _P, _P, _P], _INT),
    "tnmc3d_init_chains": ([_P, _INT, _I64, _U64, _P, _P, _P, _P], _INT),
    "tnmc3d_mh_step": ([_P, _I64, _I64, _P, _P, _P, _P, _P, _P, _U64, _U64, _P, _P, _P], _INT),
})

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_hooks = None   # keeps the ctypes callbacks alive while the library may call them


def lib():
    """Open libtnmc.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TnmcError("libtnmc.so not found at %s: run `python -m paper_2104_13264_gb300.build`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator
    (tnmc_set_allocator).  Objects created afterwards allocate and free through it."""
    import torch
    global _hooks

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:  # noqa: BLE001 -- out of memory: the library reports TNMC_E_NOMEM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().tnmc_set_allocator(ctypes.cast(hooks[0], _P), ctypes.cast(hooks[1], _P), None))
    _hooks = hooks


def use_default_allocator():
    """Back to cudaMallocAsync / cudaFreeAsync for objects created afterwards.  Objects
    created under the torch hook keep freeing through it, so its callbacks stay referenced."""
    _check(lib().tnmc_set_allocator(None, None, None))


def _check(status):
    if status != 0:
        msg = lib().tnmc_last_error().decode(errors="replace")
        raise TnmcError("tnmc status %d: %s" % (status, msg))


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Env:
    """FP64-built row environments of one instance (owned by the library).  gauge "spin"
    or "bond" (App. A's bond basis); sweeps > 0 compresses each row by that many rounds of
    two-site variational sweeps after successive SVD (spin basis only)."""

    def __init__(self, Jh, Jv, h, beta, chi, precisions=("f64",), stream=None, gauge="spin", sweeps=0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        Ly, Lx = h.shape
        Jh = np.ascontiguousarray(np.asarray(Jh, dtype=np.float64).reshape(Ly, max(Lx - 1, 0)))
        Jv = np.ascontiguousarray(np.asarray(Jv, dtype=np.float64).reshape(max(Ly - 1, 0), Lx))
        self.Lx, self.Ly, self.beta, self.chi = Lx, Ly, float(beta), int(chi)
        mask = 0
        for p in precisions:
            mask |= 1 << PRECISIONS[p]
        lat = _Lattice(Lx, Ly, Jh.ctypes.data if Jh.size else None, Jv.ctypes.data if Jv.size else None,
                       h.ctypes.data)
        out = ctypes.c_void_p()
        self._h = None
        if sweeps:
            if gauge != "spin":
                raise ValueError("variational compression is built for the spin basis only")
            _check(lib().tnmc_build_env_variational(ctypes.byref(lat), self.beta, self.chi, int(sweeps), mask,
                                                    _stream(stream), ctypes.byref(out)))
        else:
            build = {"spin": lib().tnmc_build_env, "bond": lib().tnmc_build_env_bond}[gauge]
            _check(build(ctypes.byref(lat), self.beta, self.chi, mask, _stream(stream), ctypes.byref(out)))
        self._h = out

    @classmethod
    def _wrap(cls, handle, Lx, Ly, beta, chi):
        self = cls.__new__(cls)
        self.Lx, self.Ly, self.beta, self.chi = Lx, Ly, float(beta), int(chi)
        self._h = handle
        return self

    @classmethod
    def from_instance(cls, inst, precisions=("f64",), chi=None, stream=None, gauge="spin", sweeps=0):
        return cls(inst.Jh, inst.Jv, inst.h, inst.beta, inst.chi if chi is None else chi, precisions, stream, gauge,
                   sweeps)

    @property
    def handle(self):
        return self._h

    def info(self):
        i = _Info()
        _check(lib().tnmc_env_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in _Info._fields_}

    def export(self):
        """Host copies: tensors [Ly][Lx][P][2][P], log_scale, sv, discarded, bond_dims."""
        inf = self.info()
        P, Lx, Ly = inf["pad"], self.Lx, self.Ly
        T = np.zeros((Ly, Lx, P, 2, P))
        ls = np.zeros(Ly)
        sv = np.zeros((Ly, Lx + 1, P))
        dsc = np.zeros((Ly, Lx + 1))
        bd = np.zeros((Ly, Lx + 1), dtype=np.int32)
        _check(lib().tnmc_env_export(self._h, T.ctypes.data, ls.ctypes.data, sv.ctypes.data, dsc.ctypes.data,
                                     bd.ctypes.data))
        return {"tensors": T, "log_scale": ls, "sv": sv, "discarded": dsc, "bond_dims": bd, "logZ": inf["logZ"]}

    def status(self):
        s = ctypes.c_int32()
        _check(lib().tnmc_env_status(self._h, ctypes.byref(s)))
        return s.value

    def set_order(self, order):
        """Site order of later sampling calls: "raster" or "snake" (odd rows right to left)."""
        _check(lib().tnmc_env_set_order(self._h, {"raster": 0, "snake": 1}[order]))
        return self

    def free(self):
        if self._h is not None and self._h.value:
            lib().tnmc_env_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sample(env, B, seed=0, sample_offset=0, precision="f64", out=None, stream=None):
    """Draw B proposals: returns (spins int8 [B,Ly,Lx], logq [B], energy [B], flags [B]) on cuda."""
    import torch
    dev = torch.device("cuda")
    if out is None:
        out = (torch.empty((B, env.Ly, env.Lx), dtype=torch.int8, device=dev),
               torch.empty(B, dtype=torch.float64, device=dev), torch.empty(B, dtype=torch.float64, device=dev),
               torch.empty(B, dtype=torch.int32, device=dev))
    sp, lq, E, fl = out
    _check(lib().tnmc_sample(env.handle, PRECISIONS[precision], B, seed, sample_offset, _ptr(sp), _ptr(lq),
                             _ptr(E), _ptr(fl), _stream(stream)))
    return sp, lq, E, fl


def logq(env, spins, precision="f64", stream=None):
    """Forced log q and energy of configurations spins (int8 cuda tensor [B,Ly,Lx])."""
    import torch
    spins = spins.contiguous()
    B = spins.shape[0]
    lq = torch.empty(B, dtype=torch.float64, device=spins.device)
    E = torch.empty(B, dtype=torch.float64, device=spins.device)
    fl = torch.empty(B, dtype=torch.int32, device=spins.device)
    _check(lib().tnmc_logq(env.handle, PRECISIONS[precision], B, _ptr(spins), _ptr(lq), _ptr(E), _ptr(fl),
                           _stream(stream)))
    return lq, E, fl


def init_chains(env, C, seed=0, precision="f64", stream=None):
    import torch
    dev = torch.device("cuda")
    sp = torch.empty((C, env.Ly, env.Lx), dtype=torch.int8, device=dev)
    lq = torch.empty(C, dtype=torch.float64, device=dev)
    E = torch.empty(C, dtype=torch.float64, device=dev)
    _check(lib().tnmc_init_chains(env.handle, PRECISIONS[precision], C, seed, _ptr(sp), _ptr(lq), _ptr(E),
                                  _stream(stream)))
    return sp, lq, E


def mh_step(env, C, T, prop, chain, seed=0, step_offset=0, accepted=None, n_accepted=None, stream=None):
    """MH scan; prop = (spins, logq, energy) [C*T], chain = (spins, logq, energy) [C] updated in place."""
    import torch
    ps, plq, pE = prop
    cs, clq, cE = chain
    if accepted is None:
        accepted = torch.empty(C * T, dtype=torch.uint8, device=plq.device)
    _check(lib().tnmc_mh_step(env.handle, C, T, _ptr(ps), _ptr(plq), _ptr(pE), _ptr(cs), _ptr(clq), _ptr(cE),
                              seed, step_offset, _ptr(accepted), _ptr(n_accepted), _stream(stream)))
    return accepted


def metropolis(env, chain, seed=0, chain_offset=0, sweep_offset=0, sweeps=1, precision="f64", stream=None):
    """Checkerboard Metropolis sweeps of chain = (spins, logq, energy) in place; the chains'
    log q and energy are recomputed afterwards."""
    cs, clq, cE = chain
    _check(lib().tnmc_metropolis(env.handle, PRECISIONS[precision], cs.shape[0], _ptr(cs), _ptr(clq), _ptr(cE), seed,
                                 chain_offset, sweep_offset, int(sweeps), _stream(stream)))
    return chain


def link_overlap(env, chain_spins, stream=None):
    """Link overlap of the replica pairs (2k, 2k+1): float64 cuda tensor [C / 2]."""
    import torch
    C = chain_spins.shape[0]
    out = torch.empty(C // 2, dtype=torch.float64, device=chain_spins.device)
    _check(lib().tnmc_link_overlap(env.handle, C, _ptr(chain_spins), _ptr(out), _stream(stream)))
    return out


def param_count(env):
    inf = env.info()
    return env.Ly * env.Lx * inf["pad"] * 2 * inf["pad"]


def get_params(env, stream=None):
    """FP32 sampler tensors as a flat cuda tensor [Ly*Lx*P*2*P] (a copy)."""
    import torch
    out = torch.empty(param_count(env), dtype=torch.float32, device="cuda")
    _check(lib().tnmc_env_get_params(env.handle, _ptr(out), _stream(stream)))
    return out


def set_params(env, params, stream=None):
    """Copy flat FP32 tensors into the env (the FP32 sampler then uses them)."""
    p = params.detach().contiguous()
    assert p.dtype.is_floating_point and p.numel() == param_count(env)
    _check(lib().tnmc_env_set_params(env.handle, _ptr(p.float()), _stream(stream)))


def set_tensors(env, tensors, stream=None):
    """Replace the FP64 tensors ([Ly][Lx][P][2][P], zero outside the bond dimensions; a
    float64 torch tensor on the device) and re-derive every sampler copy."""
    t = tensors.detach().contiguous()
    assert t.dtype == __import__("torch").float64 and t.is_cuda and t.numel() == param_count(env)
    _check(lib().tnmc_env_set_tensors(env.handle, _ptr(t), _stream(stream)))


def logq_backward(env, spins, weights, stream=None):
    """d/dparams of sum_b weights_b log q_b (flat FP32 cuda tensor)."""
    import torch
    spins = spins.contiguous()
    w = weights.contiguous().float()
    grad = torch.empty(param_count(env), dtype=torch.float32, device="cuda")
    _check(lib().tnmc_logq_backward(env.handle, spins.shape[0], _ptr(spins), _ptr(w), _ptr(grad), _stream(stream)))
    return grad


def _lattice_arrays(inst):
    h = np.ascontiguousarray(inst.h, dtype=np.float64)
    Ly, Lx = h.shape
    Jh = np.ascontiguousarray(np.asarray(inst.Jh, dtype=np.float64).reshape(Ly, max(Lx - 1, 0)))
    Jv = np.ascontiguousarray(np.asarray(inst.Jv, dtype=np.float64).reshape(max(Ly - 1, 0), Lx))
    return Jh, Jv, h


def build_envs_batched(insts, precisions=("f64",), stream=None):
    """Build every instance's environment in one builder launch; returns a list of Env."""
    n = len(insts)
    arrays = [_lattice_arrays(i) for i in insts]
    lats = (_Lattice * n)()
    for k, (Jh, Jv, h) in enumerate(arrays):
        Ly, Lx = h.shape
        lats[k] = _Lattice(Lx, Ly, Jh.ctypes.data if Jh.size else None, Jv.ctypes.data if Jv.size else None,
                           h.ctypes.data)
    beta = np.array([i.beta for i in insts], dtype=np.float64)
    chi = np.array([i.chi for i in insts], dtype=np.int32)
    mask = 0
    for p in precisions:
        mask |= 1 << PRECISIONS[p]
    out = (_P * n)()
    _check(lib().tnmc_build_env_batched(n, ctypes.cast(lats, _P), beta.ctypes.data, chi.ctypes.data, mask,
                                        _stream(stream), ctypes.cast(out, _P)))
    return [Env._wrap(_P(out[k]), arrays[k][2].shape[1], arrays[k][2].shape[0], insts[k].beta, insts[k].chi)
            for k in range(n)]


class Batch:
    """A plan over many envs: one persistent launch samples them all (see tnmc_batch_create).

    Keeps references to the envs, which must outlive the plan.
    """

    ORDERS = {"instance": 0, "cost": 1}

    def __init__(self, envs, B, chains=1, precision="f32", tile=128, order="cost", stream=None):
        n = len(envs)
        self.envs = list(envs)
        self.B = np.ascontiguousarray(np.broadcast_to(np.asarray(B, dtype=np.int64), (n,)))
        handles = (_P * n)(*[e.handle.value for e in self.envs])
        out = _P()
        self._h = None
        _check(lib().tnmc_batch_create(n, ctypes.cast(handles, _P), self.B.ctypes.data, int(chains),
                                       PRECISIONS[precision], int(tile), self.ORDERS[order], _stream(stream),
                                       ctypes.byref(out)))
        self._h = out
        self.n, self.chains, self.precision, self.tile, self.order = n, int(chains), precision, int(tile), order
        self.prop_row = np.zeros(n, dtype=np.int64)
        self.prop_spin = np.zeros(n, dtype=np.int64)
        self.chain_row = np.zeros(n, dtype=np.int64)
        self.chain_spin = np.zeros(n, dtype=np.int64)
        _check(lib().tnmc_batch_layout(self._h, self.prop_row.ctypes.data, self.prop_spin.ctypes.data,
                                       self.chain_row.ctypes.data, self.chain_spin.ctypes.data))

    def info(self):
        i = _BatchInfo()
        _check(lib().tnmc_batch_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in _BatchInfo._fields_}

    def alloc_proposals(self):
        """(spins arena int8, logq, energy, flags) cuda tensors for one step."""
        import torch
        inf = self.info()
        dev = torch.device("cuda")
        return (torch.empty(inf["proposal_bytes"], dtype=torch.int8, device=dev),
                torch.empty(inf["proposal_rows"], dtype=torch.float64, device=dev),
                torch.empty(inf["proposal_rows"], dtype=torch.float64, device=dev),
                torch.empty(inf["proposal_rows"], dtype=torch.int32, device=dev))

    def alloc_chains(self):
        import torch
        inf = self.info()
        dev = torch.device("cuda")
        return (torch.empty(inf["chain_bytes"], dtype=torch.int8, device=dev),
                torch.empty(inf["chain_rows"], dtype=torch.float64, device=dev),
                torch.empty(inf["chain_rows"], dtype=torch.float64, device=dev))

    def view(self, arena, i, chains=False):
        """Instance i's [rows, Ly, Lx] view of a spin arena."""
        e = self.envs[i]
        off = int(self.chain_spin[i] if chains else self.prop_spin[i])
        rows = self.chains if chains else int(self.B[i])
        return arena[off:off + rows * e.Lx * e.Ly].view(rows, e.Ly, e.Lx)

    def rows(self, arr, i, chains=False):
        off = int(self.chain_row[i] if chains else self.prop_row[i])
        rows = self.chains if chains else int(self.B[i])
        return arr[off:off + rows]

    def set_step(self, seed, step, stream=None):
        _check(lib().tnmc_batch_set_step(self._h, seed, step, _stream(stream)))

    def advance(self, stream=None):
        _check(lib().tnmc_batch_advance(self._h, _stream(stream)))

    def sample(self, out, stream=None):
        sp, lq, E, fl = out
        _check(lib().tnmc_sample_batched(self._h, _ptr(sp), _ptr(lq), _ptr(E), _ptr(fl), _stream(stream)))
        return out

    def logq(self, spins, out=None, stream=None):
        import torch
        inf = self.info()
        if out is None:
            out = (torch.empty(inf["proposal_rows"], dtype=torch.float64, device=spins.device),
                   torch.empty(inf["proposal_rows"], dtype=torch.float64, device=spins.device),
                   torch.empty(inf["proposal_rows"], dtype=torch.int32, device=spins.device))
        lq, E, fl = out
        _check(lib().tnmc_logq_batched(self._h, _ptr(spins), _ptr(lq), _ptr(E), _ptr(fl), _stream(stream)))
        return out

    def init_chains(self, seed, out=None, stream=None):
        out = self.alloc_chains() if out is None else out
        sp, lq, E = out
        _check(lib().tnmc_batch_init_chains(self._h, seed, _ptr(sp), _ptr(lq), _ptr(E), _stream(stream)))
        return out

    def mh(self, prop, chain, accepted=None, n_accepted=None, stream=None):
        ps, plq, pE = prop[:3]
        cs, clq, cE = chain
        _check(lib().tnmc_mh_batched(self._h, _ptr(ps), _ptr(plq), _ptr(pE), _ptr(cs), _ptr(clq), _ptr(cE),
                                     _ptr(accepted), _ptr(n_accepted), _stream(stream)))
        return accepted

    def metropolis(self, chain, sweeps=1, stream=None):
        """Metropolis sweeps of every chain (plan seed and step), then their log q and energy."""
        cs, clq, cE = chain
        _check(lib().tnmc_metropolis_batched(self._h, _ptr(cs), _ptr(clq), _ptr(cE), int(sweeps), _stream(stream)))
        return chain

    def link_overlap(self, chain_spins, out=None, stream=None):
        """Link overlaps of every instance's replica pairs: float64 cuda tensor [n, chains / 2]."""
        import torch
        if out is None:
            out = torch.empty((self.n, self.chains // 2), dtype=torch.float64, device=chain_spins.device)
        _check(lib().tnmc_link_overlap_batched(self._h, _ptr(chain_spins), _ptr(out), _stream(stream)))
        return out

    def balance(self):
        """(efficiency, makespan ms) of the last persistent sampling launch (tnmc_batch_balance)."""
        e, m = ctypes.c_double(), ctypes.c_double()
        _check(lib().tnmc_batch_balance(self._h, ctypes.byref(e), ctypes.byref(m)))
        return e.value, m.value

    def free(self):
        if self._h is not None and self._h.value:
            lib().tnmc_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---- three-dimensional lattices (Sec. 3D) ----

class Env3D:
    """Layer environments of a cubic-lattice instance (PEPS of bond D; the sampler's boundary
    MPS have bond chi), built by tnmc3d_build_env, or by tnmc3d_build_env_bond when
    gauge="bond" (layers sampled from their uncompressed PEPS, bond up to 2D)."""

    def __init__(self, Jx, Jy, Jz, h, beta, D, chi, stream=None, gauge="spin"):
        h = np.ascontiguousarray(h, dtype=np.float64)
        Lz, Ly, Lx = h.shape
        Jx = np.ascontiguousarray(np.asarray(Jx, dtype=np.float64).reshape(Lz, Ly, max(Lx - 1, 0)))
        Jy = np.ascontiguousarray(np.asarray(Jy, dtype=np.float64).reshape(Lz, max(Ly - 1, 0), Lx))
        Jz = np.ascontiguousarray(np.asarray(Jz, dtype=np.float64).reshape(max(Lz - 1, 0), Ly, Lx))
        self.Lz, self.Ly, self.Lx = Lz, Ly, Lx
        self.beta, self.D, self.chi = float(beta), int(D), int(chi)
        self.gauge = gauge
        self.Ds = 2 * self.D if gauge == "bond" else self.D
        lat = _Lattice3D(Lx, Ly, Lz, Jx.ctypes.data if Jx.size else None, Jy.ctypes.data if Jy.size else None,
                         Jz.ctypes.data if Jz.size else None, h.ctypes.data)
        out = ctypes.c_void_p()
        self._h = None
        build = {"spin": lib().tnmc3d_build_env, "bond": lib().tnmc3d_build_env_bond}[gauge]
        _check(build(ctypes.byref(lat), self.beta, self.D, self.chi, _stream(stream), ctypes.byref(out)))
        self._h = out

    @classmethod
    def from_instance(cls, inst, D=None, chi=None, stream=None, gauge="spin"):
        return cls(inst.Jx, inst.Jy, inst.Jz, inst.h, inst.beta, inst.D if D is None else D,
                   inst.chi if chi is None else chi, stream, gauge)

    @property
    def handle(self):
        return self._h

    @property
    def n(self):
        return self.Lz * self.Ly * self.Lx

    def export(self):
        """Host copies of the sampling tensors [Lz, Ly, Lx, 2, P, P, P, P] (P = D, or 2D in the
        bond basis), their dims [Lz, Ly, Lx, 4], and log_scale [Lz]."""
        D = self.Ds
        T = np.zeros((self.Lz, self.Ly, self.Lx, 2, D, D, D, D))
        dims = np.zeros((self.Lz, self.Ly, self.Lx, 4), dtype=np.int32)
        ls = np.zeros(self.Lz)
        _check(lib().tnmc3d_env_export(self._h, T.ctypes.data, dims.ctypes.data, ls.ctypes.data))
        return {"tensors": T, "dims": dims, "log_scale": ls}

    def status(self):
        s = ctypes.c_int32()
        _check(lib().tnmc3d_env_status(self._h, ctypes.byref(s)))
        return s.value

    def free(self):
        if self._h is not None and self._h.value:
            lib().tnmc3d_env_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sample3d(env, B, seed=0, sample_offset=0, precision="f64", stream=None):
    """Draw B proposals on a cubic lattice: (spins int8 [B,Lz,Ly,Lx], logq, energy, flags) on cuda."""
    import torch
    dev = torch.device("cuda")
    sp = torch.empty((B, env.Lz, env.Ly, env.Lx), dtype=torch.int8, device=dev)
    lq = torch.empty(B, dtype=torch.float64, device=dev)
    E = torch.empty(B, dtype=torch.float64, device=dev)
    fl = torch.empty(B, dtype=torch.int32, device=dev)
    _check(lib().tnmc3d_sample(env.handle, PRECISIONS[precision], B, seed, sample_offset, _ptr(sp), _ptr(lq), _ptr(E),
                               _ptr(fl), _stream(stream)))
    return sp, lq, E, fl


def logq3d(env, spins, precision="f64", stream=None):
    """Forced log q and energy of cubic-lattice configurations (int8 cuda tensor [B,Lz,Ly,Lx])."""
    import torch
    spins = spins.contiguous()
    B = spins.shape[0]
    lq = torch.empty(B, dtype=torch.float64, device=spins.device)
    E = torch.empty(B, dtype=torch.float64, device=spins.device)
    fl = torch.empty(B, dtype=torch.int32, device=spins.device)
    _check(lib().tnmc3d_logq(env.handle, PRECISIONS[precision], B, _ptr(spins), _ptr(lq), _ptr(E), _ptr(fl),
                             _stream(stream)))
    return lq, E, fl


def init_chains3d(env, C, seed=0, precision="f64", stream=None):
    import torch
    dev = torch.device("cuda")
    sp = torch.empty((C, env.Lz, env.Ly, env.Lx), dtype=torch.int8, device=dev)
    lq = torch.empty(C, dtype=torch.float64, device=dev)
    E = torch.empty(C, dtype=torch.float64, device=dev)
    _check(lib().tnmc3d_init_chains(env.handle, PRECISIONS[precision], C, seed, _ptr(sp), _ptr(lq), _ptr(E),
                                    _stream(stream)))
    return sp, lq, E


def mh_step3d(env, C, T, prop, chain, seed=0, step_offset=0, accepted=None, n_accepted=None, stream=None):
    """MH scan on cubic-lattice chains; as mh_step."""
    import torch
    ps, plq, pE = prop
    cs, clq, cE = chain
    if accepted is None:
        accepted = torch.empty(C * T, dtype=torch.uint8, device=plq.device)
    _check(lib().tnmc3d_mh_step(env.handle, C, T, _ptr(ps), _ptr(plq), _ptr(pE), _ptr(cs), _ptr(clq), _ptr(cE), seed,
                                step_offset, _ptr(accepted), _ptr(n_accepted), _stream(stream)))
    return accepted
