"""Thin ctypes binding of the C ABI in ``include/ddppo.h``.

Functions carry the C names; each marshals torch tensors (device memory owned by
the caller) into pointers and passes torch's current CUDA stream. All compute
runs in the CUDA library; there is no fallback path: if the library or a GPU is
missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

DDPPO_OK = 0
ERRORS = {-1: "E_ARG", -2: "E_CONFIG", -3: "E_CUDA", -4: "E_DEVICE_BOUNDS", -5: "E_TIMEOUT",
          -6: "E_STATE"}
NSTATE = 12
NSTATS = 8
NUM_ACTIONS = 4


class DDPPOError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("num_envs", ctypes.c_int32), ("gen_kind", ctypes.c_int32),
        ("grid_min", ctypes.c_int32), ("grid_max", ctypes.c_int32),
        ("cell_m", ctypes.c_float), ("wall_density", ctypes.c_float),
        ("door_m", ctypes.c_float), ("min_room", ctypes.c_int32),
        ("max_steps", ctypes.c_int32), ("terminal_mode", ctypes.c_int32),
        ("depth_h", ctypes.c_int32), ("depth_w", ctypes.c_int32),
        ("pool2x2", ctypes.c_int32), ("cam_h_m", ctypes.c_float),
        ("ceil_h_m", ctypes.c_float), ("max_depth_m", ctypes.c_float),
        ("net_kind", ctypes.c_int32), ("base_ch", ctypes.c_int32),
        ("hidden", ctypes.c_int32), ("lstm_layers", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("rollout_T", ctypes.c_int32),
        ("minibatches", ctypes.c_int32), ("encoder_chunk", ctypes.c_int32),
        ("task", ctypes.c_int32), ("explore_m", ctypes.c_float),
        ("seed", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Rollout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "obs", "goal", "prev_a", "masks", "actions", "logp", "values", "rewards", "dones", "info",
        "adv", "ret", "h0", "c0", "h", "c", "uniforms")]


class PPOHParams(ctypes.Structure):
    _fields_ = [
        ("clip", ctypes.c_float), ("lr", ctypes.c_float), ("value_coef", ctypes.c_float),
        ("entropy_coef", ctypes.c_float), ("max_grad_norm", ctypes.c_float),
        ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
        ("epochs", ctypes.c_int32), ("minibatches", ctypes.c_int32),
        ("norm_adv", ctypes.c_int32), ("update_index", ctypes.c_int32),
    ]


def default_hparams(**kw) -> PPOHParams:
    """Sec. 4 "Training": 2 epochs x 2 minibatches, Adam 2.5e-4, no advantage norm."""
    d = dict(clip=0.2, lr=2.5e-4, value_coef=0.5, entropy_coef=0.01, max_grad_norm=0.5,
             beta1=0.9, beta2=0.999, adam_eps=1e-5, epochs=2, minibatches=2, norm_adv=0,
             update_index=0)
    d.update(kw)
    return PPOHParams(**d)


_lib = None
P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F32 = ctypes.c_float

_SIGS = {
    "ddppo_create": [P, P],
    "ddppo_config_check": [P],
    "ddppo_destroy": [P],
    "ddppo_device_status": [P, P, P],
    "ddppo_set_bfs_level_cap": [P, I32],
    "ddppo_num_params": [P, P],
    "ddppo_get_params": [P, P, I64, P],
    "ddppo_set_params": [P, P, I64, P],
    "ddppo_get_adam": [P, P, P, I64, P, P],
    "ddppo_env_reset": [P, P, P, P],
    "ddppo_env_step": [P, P, P, P, P, P, P, P],
    "ddppo_env_prefetch": [P, P],
    "ddppo_env_state": [P, P, P],
    "ddppo_env_set_state": [P, P, P],
    "ddppo_env_grids": [P, P, P, P],
    "ddppo_env_depth": [P, P, P],
    "ddppo_policy_act": [P, P, P, P, P, P, P, P, P, P, P, P],
    "ddppo_policy_evaluate": [P, I32, I32, P, P, P, P, P, P, P, P, P],
    "ddppo_policy_backward": [P, P, P, P, P],
    "ddppo_encoder_forward": [P, I32, P, P, P],
    "ddppo_encoder_backward": [P, P, P, P],
    "ddppo_lstm_forward": [P, I32, I32, P, P, P, P, P, P],
    "ddppo_lstm_backward": [P, P, P, P, P],
    "ddppo_gae": [P, P, P, I32, I32, F32, F32, P, P, P],
    "ddppo_ppo_loss": [I32, P, P, P, P, P, P, F32, F32, F32, P, P, P, P],
    "ddppo_ppo_loss_static": [I32, P, P, P, P, P, P, F32, F32, F32, P, P, P, P],
    "ddppo_ppo_update": [P, P, P, P, P],
    "ddppo_collect": [P, P, I32, P],
    "ddppo_collect_begin": [P, P, P],
    "ddppo_collect_step": [P, P, I32, P],
    "ddppo_collect_end": [P, P, I32, P],
    "ddppo_ppo_grad": [P, P, P, I32, I32, I32, P, P, P],
    "ddppo_apply_grad": [P, P, F32, P, P, P],
    "ddppo_grad_mean": [I32, P, I64, P, P],
    "ddppo_save": [P, P, ctypes.c_char_p, P],
    "ddppo_load": [P, P, ctypes.c_char_p, P],
    "ddppo_timing_enable": [P, I32],
    "ddppo_timing_read": [P, I32, P, P, P],
    "ddppo_count_kernels": [P, P, P, F32, F32, P],
    "ddppo_gemm": [I32, I32, I32, I32, P, I32, I32, P, I32, I32, P, I32, I32, F32, P, I32, P, P],
    "ddppo_gemm_backend": [I32, I32, I32, I32, P, I32, P, I32, P],
    "ddppo_timing_launches": [P, I32, P, P, P, I64, P],
    "ddppo_autotune": [P, I32, P],
    "ddppo_lstm_whole_segment": [P, I32],
    "ddppo_group_norm_one_launch": [P, I32],
    "ddppo_update_graph": [P, I32],
    "ddppo_set_launch_overlap": [I32],
    "ddppo_launch_overlap": [P],
    "ddppo_set_tma_epilogue": [I32],
    "ddppo_tma_epilogue": [P],
    "ddppo_autotune_export": [P, P, ctypes.c_size_t, P],
    "ddppo_autotune_import": [P, P, ctypes.c_size_t],
    "ddppo_conv2d": [I32, I32, I32, I32, I32, I32, I32, I32, P, P, P, F32, P, P],
    "ddppo_conv2d_wgrad": [I32, I32, I32, I32, I32, I32, I32, I32, P, P, P, F32, P, P],
    "ddppo_quantize_e4m3": [P, I32, I64, P, P, P],
    "ddppo_conv_plan": [I32, I32, I32, I32, I32, I32, I32, I32, P],
    "ddppo_group_norm": [I32, I32, I32, P, P, P, P, I32, P, P, P, P],
    "ddppo_grouped_conv3x3": [I32, I32, I32, I32, I32, I32, P, P, P, P],
    "ddppo_squeeze_excite": [I32, I32, I32, I32, P, P, P, P, P, P, P, P, P, P, P],
    "ddppo_gemm_e4m3": [I32, I32, I32, P, I32, P, I32, P, P, P, I32, F32, P, I32, P, P],
    "ddppo_conv2d_e4m3": [I32, I32, I32, I32, I32, I32, I32, I32, P, P, P, P, P, F32, P, P],
}


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.ddppo_last_error.restype = ctypes.c_char_p
        L.ddppo_last_error.argtypes = []
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS) + ["ddppo_last_error"]


def _check(rc: int):
    if rc != DDPPO_OK:
        raise DDPPOError(rc, lib().ddppo_last_error().decode())


def _p(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _s(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---- thin wrappers with the C names ----
def ddppo_create(cfg: Config):
    h = ctypes.c_void_p()
    _check(lib().ddppo_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def ddppo_destroy(h):
    _check(lib().ddppo_destroy(h))


def ddppo_config_check(cfg) -> None:
    """Raise DDPPOError when ddppo_create would reject cfg (host only, no GPU needed)."""
    _check(lib().ddppo_config_check(ctypes.byref(cfg)))


def ddppo_device_status(h) -> int:
    code = ctypes.c_int32()
    _check(lib().ddppo_device_status(h, ctypes.byref(code), _s()))
    return code.value


def ddppo_set_bfs_level_cap(h, cap: int) -> None:
    """Cap the BFS level loop (0 restores the default); a test setting, see the header."""
    _check(lib().ddppo_set_bfs_level_cap(h, cap))


def ddppo_num_params(h) -> int:
    n = ctypes.c_int64()
    _check(lib().ddppo_num_params(h, ctypes.byref(n)))
    return n.value


def ddppo_get_params(h, flat):
    _check(lib().ddppo_get_params(h, _p(flat), flat.numel(), _s()))


def ddppo_set_params(h, flat):
    _check(lib().ddppo_set_params(h, _p(flat), flat.numel(), _s()))


def ddppo_get_adam(h, m, v) -> int:
    step = ctypes.c_int64()
    _check(lib().ddppo_get_adam(h, _p(m), _p(v), m.numel(), ctypes.byref(step), _s()))
    return step.value


def ddppo_env_reset(h, obs, goal):
    _check(lib().ddppo_env_reset(h, _p(obs), _p(goal), _s()))


def ddppo_env_step(h, actions, obs, goal, reward, done, info=None):
    _check(lib().ddppo_env_step(h, _p(actions), _p(obs), _p(goal), _p(reward), _p(done), _p(info),
                                _s()))


def ddppo_env_prefetch(h, stream=None):
    """Prepare the next episode of every env (see the header); stream: a torch stream."""
    _check(lib().ddppo_env_prefetch(h, _s(stream)))


def ddppo_env_state(h, state):
    _check(lib().ddppo_env_state(h, _p(state), _s()))


def ddppo_env_set_state(h, state):
    _check(lib().ddppo_env_set_state(h, _p(state), _s()))


def ddppo_env_grids(h, grids=None, dists=None):
    _check(lib().ddppo_env_grids(h, _p(grids), _p(dists), _s()))


def ddppo_env_depth(h, depth):
    _check(lib().ddppo_env_depth(h, _p(depth), _s()))


def ddppo_policy_act(h, obs, goal, prev_a, masks, hs, cs, uniforms, action, logp, value):
    _check(lib().ddppo_policy_act(h, _p(obs), _p(goal), _p(prev_a), _p(masks), _p(hs), _p(cs),
                                  _p(uniforms), _p(action), _p(logp), _p(value), _s()))


def ddppo_policy_evaluate(h, T, E, obs, goal, prev_a, masks, h0, c0, logits, values):
    _check(lib().ddppo_policy_evaluate(h, T, E, _p(obs), _p(goal), _p(prev_a), _p(masks), _p(h0),
                                       _p(c0), _p(logits), _p(values), _s()))


def ddppo_policy_backward(h, dlogits, dvalues, grad):
    _check(lib().ddppo_policy_backward(h, _p(dlogits), _p(dvalues), _p(grad), _s()))


def ddppo_encoder_forward(h, N, obs, feat):
    _check(lib().ddppo_encoder_forward(h, N, _p(obs), _p(feat), _s()))


def ddppo_encoder_backward(h, dfeat, grad):
    _check(lib().ddppo_encoder_backward(h, _p(dfeat), _p(grad), _s()))


def ddppo_lstm_forward(h, T, E, x, masks, h0, c0, y):
    _check(lib().ddppo_lstm_forward(h, T, E, _p(x), _p(masks), _p(h0), _p(c0), _p(y), _s()))


def ddppo_lstm_backward(h, dy, dx, grad):
    _check(lib().ddppo_lstm_backward(h, _p(dy), _p(dx), _p(grad), _s()))


def ddppo_gae(reward, done, value, T, E, gamma, lam, adv, ret):
    _check(lib().ddppo_gae(_p(reward), _p(done), _p(value), T, E, gamma, lam, _p(adv), _p(ret),
                           _s()))


def ddppo_ppo_loss(n, logits, values, actions, logp_old, adv, ret, clip, value_coef, entropy_coef,
                   stats, dlogits, dvalues):
    _check(lib().ddppo_ppo_loss(n, _p(logits), _p(values), _p(actions), _p(logp_old), _p(adv),
                                _p(ret), clip, value_coef, entropy_coef, _p(stats), _p(dlogits),
                                _p(dvalues), _s()))


def ddppo_ppo_loss_static(n, logits, values, actions, logp_old, adv, ret, clip, value_coef,
                          entropy_coef, stats, dlogits, dvalues):
    _check(lib().ddppo_ppo_loss_static(n, _p(logits), _p(values), _p(actions), _p(logp_old),
                                       _p(adv), _p(ret), clip, value_coef, entropy_coef,
                                       _p(stats), _p(dlogits), _p(dvalues), _s()))


def ddppo_ppo_update(h, ro: Rollout, hp: PPOHParams, stats=None):
    _check(lib().ddppo_ppo_update(h, ctypes.byref(ro), ctypes.byref(hp), _p(stats), _s()))


def ddppo_collect(h, ro: Rollout, use_graph: bool = True):
    _check(lib().ddppo_collect(h, ctypes.byref(ro), 1 if use_graph else 0, _s()))


def ddppo_collect_begin(h, ro: Rollout, stream=None):
    _check(lib().ddppo_collect_begin(h, ctypes.byref(ro), _s(stream)))


def ddppo_collect_step(h, ro: Rollout, t: int, stream=None):
    _check(lib().ddppo_collect_step(h, ctypes.byref(ro), t, _s(stream)))


def ddppo_collect_end(h, ro: Rollout, T_valid: int, stream=None):
    _check(lib().ddppo_collect_end(h, ctypes.byref(ro), T_valid, _s(stream)))


def ddppo_ppo_grad(h, ro: Rollout, hp: PPOHParams, T_valid: int, epoch: int, k: int, grad,
                   stats=None, stream=None):
    _check(lib().ddppo_ppo_grad(h, ctypes.byref(ro), ctypes.byref(hp), T_valid, epoch, k, _p(grad),
                                _p(stats), _s(stream)))


def ddppo_apply_grad(h, grad, scale: float, hp: PPOHParams, stats=None, stream=None):
    _check(lib().ddppo_apply_grad(h, _p(grad), scale, ctypes.byref(hp), _p(stats), _s(stream)))


def ddppo_grad_mean(bufs, out, stream=None):
    """out = mean of the equally sized CUDA tensors in bufs (fixed summation order)."""
    arr = (ctypes.c_void_p * len(bufs))(*[b.data_ptr() for b in bufs])
    _check(lib().ddppo_grad_mean(len(bufs), arr, out.numel(), _p(out), _s(stream)))


def ddppo_save(h, path: str, ro: Rollout | None = None):
    """Checkpoint the worker (and, with ro, the rollout state the next collect carries)."""
    _check(lib().ddppo_save(h, ctypes.byref(ro) if ro is not None else None,
                            os.fsencode(path), _s()))


def ddppo_load(h, path: str, ro: Rollout | None = None):
    """Restore a checkpoint written by ddppo_save for a worker of the same configuration."""
    _check(lib().ddppo_load(h, ctypes.byref(ro) if ro is not None else None,
                            os.fsencode(path), _s()))


def ddppo_timing_enable(h, on: bool):
    _check(lib().ddppo_timing_enable(h, 1 if on else 0))


def ddppo_timing_read(h, family: int):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    w = ctypes.c_double()
    _check(lib().ddppo_timing_read(h, family, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
    return ms.value, n.value, w.value


def ddppo_count_kernels(h, ro: Rollout, hp: PPOHParams, gamma: float, lam: float) -> int:
    n = ctypes.c_int64()
    _check(lib().ddppo_count_kernels(h, ctypes.byref(ro), ctypes.byref(hp), gamma, lam,
                                     ctypes.byref(n)))
    return n.value


def ddppo_gemm(A, B, C, beta=0.0, bias=None, relu=False, status=None, M=None, N=None, K=None,
               lda=None, ldb=None, ldc=None, a_t=False, b_t=False):
    """C = beta*C + A @ B^T (+ bias) (ReLU) on the library's GEMM (bf16 operands -> tcgen05).
    With a_t the tensor A holds A^T ([K, M]); with b_t B holds B^T ([K, N])."""
    M = (A.shape[1] if a_t else A.shape[0]) if M is None else M
    N = (B.shape[1] if b_t else B.shape[0]) if N is None else N
    K = (A.shape[0] if a_t else A.shape[1]) if K is None else K
    lda = A.stride(0) if lda is None else lda
    ldb = B.stride(0) if ldb is None else ldb
    ldc = C.stride(0) if ldc is None else ldc
    op_bf16 = 1 if A.dtype == torch.bfloat16 else 0
    _check(lib().ddppo_gemm(M, N, K, op_bf16, ctypes.c_void_p(A.data_ptr()), lda, 1 if a_t else 0,
                            ctypes.c_void_p(B.data_ptr()), ldb, 1 if b_t else 0,
                            ctypes.c_void_p(C.data_ptr()), ldc,
                            1 if C.dtype == torch.bfloat16 else 0, beta, _p(bias),
                            1 if relu else 0, _p(status), _s()))


def ddppo_gemm_backend(A, B) -> bool:
    t = ctypes.c_int32()
    _check(lib().ddppo_gemm_backend(A.shape[0], B.shape[0], A.shape[1],
                                    1 if A.dtype == torch.bfloat16 else 0,
                                    ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                    ctypes.c_void_p(B.data_ptr()), B.stride(0), ctypes.byref(t)))
    return bool(t.value)


def ddppo_timing_launches(h, family: int):
    """Per-launch (ms, work, bytes) lists of the timed launches of a kernel family."""
    n = ctypes.c_int64()
    _check(lib().ddppo_timing_launches(h, family, None, None, None, 0, ctypes.byref(n)))
    cap = n.value
    ms = (ctypes.c_double * max(cap, 1))()
    wk = (ctypes.c_double * max(cap, 1))()
    by = (ctypes.c_double * max(cap, 1))()
    _check(lib().ddppo_timing_launches(h, family, ms, wk, by, cap, ctypes.byref(n)))
    return list(ms)[:cap], list(wk)[:cap], list(by)[:cap]


def ddppo_update_graph(h, on: bool = True) -> None:
    _check(lib().ddppo_update_graph(h, 1 if on else 0))


def ddppo_lstm_whole_segment(h, mode: int = 1) -> None:
    """LSTM recurrence mode: 0 step by step (the default), 1 whole segment on CUDA cores,
    2 tcgen05 forward; a bool selects 1 (True) or 0 (False)."""
    _check(lib().ddppo_lstm_whole_segment(h, int(mode)))


def ddppo_set_launch_overlap(on: bool = True) -> None:
    _check(lib().ddppo_set_launch_overlap(1 if on else 0))


def ddppo_launch_overlap() -> bool:
    v = ctypes.c_int32()
    _check(lib().ddppo_launch_overlap(ctypes.byref(v)))
    return bool(v.value)


def ddppo_set_tma_epilogue(on: bool = True) -> None:
    _check(lib().ddppo_set_tma_epilogue(1 if on else 0))


def ddppo_tma_epilogue() -> bool:
    v = ctypes.c_int32()
    _check(lib().ddppo_tma_epilogue(ctypes.byref(v)))
    return bool(v.value)


def ddppo_group_norm_one_launch(h, on: bool = True) -> None:
    _check(lib().ddppo_group_norm_one_launch(h, 1 if on else 0))


def ddppo_autotune(h, on: bool = True) -> int:
    n = ctypes.c_int64()
    _check(lib().ddppo_autotune(h, 1 if on else 0, ctypes.byref(n)))
    return n.value


def ddppo_autotune_export(h) -> bytes:
    """The autotuner's table as a byte image (a tuning cache)."""
    n = ctypes.c_size_t()
    _check(lib().ddppo_autotune_export(h, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().ddppo_autotune_export(h, buf, n.value, ctypes.byref(n)))
    return buf.raw[:n.value]


def ddppo_autotune_import(h, image: bytes) -> None:
    buf = ctypes.create_string_buffer(bytes(image), len(image))
    _check(lib().ddppo_autotune_import(h, buf, len(image)))


def ddppo_conv_plan(N: int, H: int, W: int, C: int, Cout: int, k: int, stride: int,
                    pad: int) -> list[int]:
    """Paths and staging geometry of a bf16 convolution and its weight gradient (18 ints;
    see the header). Host only: works without a GPU."""
    plan = (ctypes.c_int32 * 18)()
    _check(lib().ddppo_conv_plan(N, H, W, C, Cout, k, stride, pad, plan))
    return list(plan)


def ddppo_quantize_e4m3(x, q, scale):
    """Per-tensor E4M3 quantisation: scale[0] = amax|x| / 448 (1 when x is all zero),
    q = e4m3(x / scale) as uint8 codes. x fp32 or bf16 (any shape), q uint8 (same numel),
    scale fp32 [1]; all CUDA tensors."""
    assert q.dtype == torch.uint8 and q.numel() == x.numel()
    _check(lib().ddppo_quantize_e4m3(_p(x), 1 if x.dtype == torch.bfloat16 else 0, x.numel(),
                                     _p(q), _p(scale), _s()))


def ddppo_gemm_e4m3(A, B, C, scale_a=None, scale_b=None, beta: float = 0.0, bias=None,
                    relu: bool = False, status=None):
    """C (+)= scale_a scale_b A B^T with A [M, K], B [N, K] E4M3 codes (uint8 or
    torch.float8_e4m3fn), C fp32 [M, N]; scales fp32 [1] CUDA tensors or None."""
    M, K = A.shape
    N = B.shape[0]
    _check(lib().ddppo_gemm_e4m3(M, N, K, _p(A), A.stride(0), _p(B), B.stride(0), _p(scale_a),
                                 _p(scale_b), _p(C), C.stride(0), beta, _p(bias), 1 if relu else 0,
                                 _p(status), _s()))


def ddppo_conv2d_e4m3(x, w, y, k: int, stride: int, pad: int, scale_x=None, scale_w=None,
                      beta: float = 0.0, status=None):
    """y = beta y + scale_x scale_w conv(x, w): x NHWC E4M3 [N, H, W, C], w E4M3
    [Cout, k*k*C] (K ordered ky, kx, c), y fp32 [N, Ho, Wo, Cout]."""
    N, H, W, C = x.shape
    _check(lib().ddppo_conv2d_e4m3(N, H, W, C, w.shape[0], k, stride, pad, _p(x), _p(w),
                                   _p(scale_x), _p(scale_w), _p(y), beta, _p(status), _s()))


def ddppo_conv2d_wgrad(x, dy, dw, k: int, stride: int, pad: int, beta: float = 0.0, status=None):
    """dw (+)= the weight gradient of conv(x, w) for output gradient dy, on the implicit
    weight-gradient path. x NHWC bf16 [N, H, W, C]; dy bf16 [N, Ho, Wo, Cout];
    dw fp32 [Cout, k*k*C] (K ordered ky, kx, c)."""
    N, H, W, C = x.shape
    _check(lib().ddppo_conv2d_wgrad(N, H, W, C, dy.shape[3], k, stride, pad, _p(x), _p(dy), _p(dw),
                                    beta, _p(status), _s()))


def ddppo_conv2d(x, w, y, k: int, stride: int, pad: int, beta: float = 0.0, status=None):
    """y = beta y + conv(x, w) on the implicit-im2col tensor-core path. x NHWC bf16
    [N, H, W, C]; w bf16 [Cout, k*k*C] (K ordered ky, kx, c); y fp32 [N, Ho, Wo, Cout]."""
    N, H, W, C = x.shape
    _check(lib().ddppo_conv2d(N, H, W, C, w.shape[0], k, stride, pad, _p(x), _p(w), _p(y),
                              beta, _p(status), _s()))


def ddppo_group_norm(z, gamma, beta, out, mean, rstd, resid=None, relu=False):
    """out = act(GroupNorm(z) + resid), C/2 groups; z, out, resid fp32 [N, HW, C]."""
    N, HW, C = z.shape
    _check(lib().ddppo_group_norm(N, HW, C, _p(z), _p(gamma), _p(beta), _p(resid), 1 if relu else 0,
                                  _p(out), _p(mean), _p(rstd), _s()))


def ddppo_grouped_conv3x3(x, w, z, groups: int, stride: int):
    """z = grouped 3x3 convolution (padding 1) of NHWC fp32 x with w [C, C/groups, 3, 3]."""
    N, H, W, C = x.shape
    _check(lib().ddppo_grouped_conv3x3(N, H, W, C, groups, stride, _p(x), _p(w), _p(z), _s()))


def ddppo_squeeze_excite(u, W1, b1, W2, b2, m, a, gate, y, sc=None):
    """Squeeze-excite of u [N, HW, C] (fp32) with the shortcut sc; see the header."""
    N, HW, C = u.shape
    _check(lib().ddppo_squeeze_excite(N, HW, C, W1.shape[0], _p(u), _p(sc), _p(W1), _p(b1), _p(W2),
                                      _p(b2), _p(m), _p(a), _p(gate), _p(y), _s()))
