"""The float32 OpenMP CPU baseline (oracle/cpu_fp32.cpp): build and call.

TEST AND BENCHMARK INFRASTRUCTURE ONLY (see the package docstring). The
benchmark times it as the fair CPU baseline on all host cores; a host test
checks it against the float64 oracle. It is compiled with the host compiler
(no architecture-specific flags, so it builds the same on x86 and Arm).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_fp32.cpp")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libcpu_fp32.so")


class Cam(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("pos", C.c_float * 3),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("znear", C.c_float), ("W", C.c_int32), ("H", C.c_int32)]


def build(force: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > os.path.getmtime(SRC):
        return LIB
    cmd = ["g++", "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c++17", "-o", LIB + ".tmp", SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"g++ failed on {SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        P = C.c_void_p
        lib.cpu_iteration.restype = C.c_int
        lib.cpu_iteration.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, C.c_int32, P,
                                      C.c_int32, P, P, P, P, C.c_int32]
        lib.cpu_adam.restype = None
        lib.cpu_adam.argtypes = [P, P, P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                 C.c_float, C.c_float, C.c_float, C.c_int32]
        _lib = lib
    return _lib


def rows_of(scene: Dict[str, np.ndarray], sh_degree: int) -> np.ndarray:
    """Parameter rows [n][stride] (mean, opacity logit, log-scale, pad,
    quaternion, SH coefficient-major; stride 16/24/40/64 for degree 0-3)."""
    n = scene["means"].shape[0]
    k = (sh_degree + 1) ** 2
    stride = {0: 16, 1: 24, 2: 40, 3: 64}[sh_degree]
    rows = np.zeros((n, stride), np.float32)
    rows[:, 0:3] = scene["means"]
    rows[:, 3] = scene["opacity_logits"]
    rows[:, 4:7] = scene["log_scales"]
    rows[:, 8:12] = scene["quats"]
    rows[:, 12:12 + 3 * k] = np.asarray(scene["sh"], np.float32)[:, :k, :].reshape(n, 3 * k)
    return rows


def cams_of(cams: Sequence) -> C.Array:
    out = (Cam * len(cams))()
    for j, c in enumerate(cams):
        R = np.asarray(c["R"], np.float64).reshape(9)
        for i in range(9):
            out[j].R[i] = float(R[i])
        for i in range(3):
            out[j].t[i] = float(c["t"][i])
            out[j].pos[i] = float(c["pos"][i])
        out[j].fx, out[j].fy = float(c["fx"]), float(c["fy"])
        out[j].cx, out[j].cy = float(c["cx"]), float(c["cy"])
        out[j].znear = float(c["znear"])
        out[j].W, out[j].H = int(c["width"]), int(c["height"])
    return out


class Baseline:
    """One scene and its views on the CPU: `iteration()` runs forward,
    backward and masked Adam; `gradients()` forward and backward only."""

    def __init__(self, scene, cams, sh_degree: int, targets, active, loss: str = "l1",
                 threads: int = 0):
        self.lib = load()
        self.deg = sh_degree
        self.rows = rows_of(scene, sh_degree)
        self.n, self.stride = self.rows.shape
        self.m = np.zeros_like(self.rows)
        self.v = np.zeros_like(self.rows)
        self.grads = np.zeros_like(self.rows)
        self.step = 0
        self.cams = cams_of(cams)
        self.V = len(cams)
        self.targets = np.ascontiguousarray(
            np.concatenate([np.asarray(t, np.float32).reshape(-1) for t in targets]))
        self.active = np.ascontiguousarray(np.asarray(active, np.uint8))
        self.loss_mode = {"l1": 1, "l2": 2}[loss]
        self.threads = int(threads)
        self.shapes = [(int(c["height"]), int(c["width"])) for c in cams]

    def gradients(self, held: Optional[Sequence[np.ndarray]] = None, want_image=False):
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        h = None
        if held is not None:
            h = np.ascontiguousarray(
                np.concatenate([np.asarray(x, np.uint8).reshape(-1) for x in held]))
        img = np.empty_like(self.targets) if want_image else None
        loss = C.c_double(0.0)
        rc = self.lib.cpu_iteration(ptr(self.rows), self.n, self.stride, self.deg,
                                    ptr(self.active), C.cast(self.cams, C.c_void_p), self.V,
                                    ptr(self.targets), self.loss_mode,
                                    None if h is None else ptr(h), ptr(self.grads),
                                    None if img is None else ptr(img), C.byref(loss),
                                    self.threads)
        if rc != 0:
            raise ValueError("cpu_iteration rejected its arguments")
        out = {"grads": self.grads, "loss": loss.value}
        if want_image:
            views, o = [], 0
            for (H, W) in self.shapes:
                views.append(img[o: o + 3 * H * W].reshape(3, H, W))
                o += 3 * H * W
            out["image"] = views
        return out

    def iteration(self, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-15) -> float:
        r = self.gradients()
        self.step += 1
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)
        self.lib.cpu_adam(ptr(self.rows), ptr(self.m), ptr(self.v), ptr(self.grads),
                          ptr(self.active), self.n, self.stride, self.step, lr, beta1, beta2,
                          eps, self.threads)
        return r["loss"]
