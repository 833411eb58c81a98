"""FP64 CPU oracle of the batched drone physics step (Crazyflow, arXiv 2606.01478).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: it is used by ``tests/``, by ``__graft_entry__.smoke()``
(to check one small GPU invocation) and by ``bench.py``'s ``cpu_baseline`` leg
and ``--impl reference`` arm.  It shares no code with the CUDA path; the only
module both sides use is ``workloads`` (seeded inputs, no method arithmetic).

The oracle is written from the paper, in float64, with plain vectorised
PyTorch CPU operations over a leading batch dimension (one row per drone) and
Python loops over time steps.  Gradients are those of this exact discrete
computation, taken by torch.autograd (a library primitive serving as the
reverse sweep), and are pinned against central finite differences.

Modules
    rotation   quaternion / Euler-angle rotations (scalar-last quaternion)
    physics    first-principles and abstracted derivatives, rotor model,
               controllers, mixer, Euler / RK4 step, rollouts
    policy     policy MLP (bf16 weights as exact float64 values), figure-8
               tracking loss and its gradient (BPTT)
    sampling   Philox4x32-10, Box-Muller, sampled rollout cost

Parity status per function is listed in each module header.  Functions whose
definitions are readings of the paper adopted here (the controller gains and structure,
the action mapping, the policy, the sampling cost) follow no printed equation
of the paper: they are "parity unpinned" against the paper and pinned only by
invariants (hover fixed point, small-angle linearisation, closed-loop
convergence, brute force on tiny inputs).
"""
