"""The AP energy as a differentiable function of positions and homogeneous strain.

E(x, eps) is the energy of the configuration x' = x (I + eps)^T in the box h' = h (I + eps)^T
(Sec. 2.2.3, Eq. energy_hyb, with the EAM and ACE terms of Secs. 2.2.1-2.2.2).  The forward
pass is one library force evaluation (kernels only); the backward pass needs no second
evaluation, because the force kernels already produced the adjoint:

    dE/dx_i   = -F'_i (I + eps)           (F' the forces of the strained configuration)
    dE/deps   = -W' (I + eps)^-T          (W' its virial, -sum r_ij (x) dE_i/dr_ij)

The energy is returned in FP64 whatever the input dtype (it is an FP64 reduction of the
per-atom energies on the device); the gradients come back in the dtypes of the inputs.

The strain derivative treats w as fixed per atom, so contexts used with a strain must have a
constant or explicit weight and no indenter (position-dependent external fields are not part
of the homogeneous-deformation identity).
"""
import numpy as np
import torch

__all__ = ["ap_energy"]


def _virial_matrix(v6, device):
    xx, yy, zz, xy, xz, yz = (float(t) for t in v6)
    return torch.tensor([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]], dtype=torch.float64, device=device)


class _APEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, positions, strain, apctx, box):
        dev = positions.device
        Fm = torch.eye(3, dtype=torch.float64, device=dev) + strain.detach().to(torch.float64)
        xs = (positions.detach().to(torch.float64) @ Fm.T).contiguous()
        h0 = torch.as_tensor(np.asarray(box["h"], dtype=np.float64).reshape(3, 3), device=dev)
        h = (h0 @ Fm.T).cpu().numpy()
        apctx.set_box({"h": h.ravel(), "origin": box.get("origin", (0.0, 0.0, 0.0)), "periodic": box["periodic"]})
        forces = torch.empty(xs.shape, dtype=torch.float32, device=dev)
        apctx.compute_forces(xs, forces)
        rep = apctx.energy()
        W = _virial_matrix(rep["virial"], dev)
        fctx.save_for_backward(forces, Fm, W)
        fctx.dtypes = (positions.dtype, strain.dtype)
        return torch.tensor(rep["e_total"], dtype=torch.float64, device=dev)

    @staticmethod
    def backward(fctx, gE):
        forces, Fm, W = fctx.saved_tensors
        g = gE.to(torch.float64)
        gx = -(forces.to(torch.float64) @ Fm) * g
        gs = -(W @ torch.linalg.inv(Fm).T) * g
        return gx.to(fctx.dtypes[0]), gs.to(fctx.dtypes[1]), None, None


def ap_energy(positions, strain, apctx, box):
    """Energy of `apctx` at `positions` ((n, 3) CUDA tensor) strained by `strain` ((3, 3)),
    with `box` the unstrained box dict; differentiable in positions and strain."""
    return _APEnergy.apply(positions, strain, apctx, box)
