"""Helpers shared by the GPU parity tests: build the same grid for the CUDA
path and the oracle, move f between them, compare."""
import numpy as np

import oracle as O
from paper_1702_08521_gb300 import vlasov as V


def both(grid: dict, precision: int):
    """(Simulation on the GPU, oracle Grid) for one grid description."""
    sim = V.Simulation(grid, precision=precision)
    og = O.grid(**grid)
    return sim, og


def to_gpu(sim, f_np: np.ndarray) -> None:
    sim.upload(f_np.reshape(-1))


def from_gpu(sim) -> np.ndarray:
    sim.sync()
    return sim.f.detach().cpu().numpy().astype(np.float64)


def snapshot(sim):
    """Copy of f once the library's queued work on it has finished."""
    import torch
    sim.sync()
    s = sim.f.clone()
    torch.cuda.synchronize()
    return s


def rel_max(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l1(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300))


def accel_tensor(sim, acc_np: np.ndarray):
    import torch
    return torch.as_tensor(np.ascontiguousarray(acc_np, dtype=np.float64).reshape(-1),
                           device=sim.f.device)
