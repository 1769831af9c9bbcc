"""The genotype-shaped bridged job (the benchmark step), parameterised by size.

Slot j of every ciphertext is one (individual, target) pair.  Per class c
the SecureMod score is sum over tags of weight[c, tag, target] x
genotype[tag, individual, target] (public weights: plaintext-vector
multiplies, then an addition tree), then the bridge SecureMod ->
SecureUint<s> (Eq. 2 / Listings 7-8) turns each score into s encrypted
bits, a levelised 3-way argmax circuit picks the best class per slot (ties
to the lower index), and the two index bits are decrypted.
"""

import numpy as np

from . import circuits, inputs

PAPER, SELECT = 0, 1


def genotype_inputs(seed, N, n_ind=8, n_targets=2000, n_tags=32, n_classes=3, wmax=64):
    """Tag genotypes [n_tags][N] and weights [n_classes][n_tags][N] (slots beyond n_ind*n_targets zero)."""
    used = n_ind * n_targets
    assert used <= N
    G = inputs.genotypes(seed, n_ind, n_targets, n_tags)
    W = inputs.weights(seed + 1, n_classes, n_tags, n_targets, n_ind) % wmax
    Gs = np.zeros((n_tags, N), dtype=np.int64)
    Ws = np.zeros((n_classes, n_tags, N), dtype=np.int64)
    Gs[:, :used] = G
    Ws[:, :, :used] = W
    return Gs, Ws


class GenotypeJob:
    def __init__(self, ctx, n_tags=32, n_classes=3, s_bits=12, mode=PAPER):
        assert n_classes == 3 and n_tags & (n_tags - 1) == 0
        self.ctx, self.n_tags, self.n_classes, self.s = ctx, n_tags, n_classes, s_bits
        self.mode = mode
        net = circuits.Netlist()
        s0, s1, s2 = net.inputs(s_bits), net.inputs(s_bits), net.inputs(s_bits)
        self.out_wires = net.argmax3(s0, s1, s2)
        self.circ = circuits.Compiled(ctx, net, 1)
        self.circuit_muls = net.n_mul
        self.last = {}

    def muls_per_run(self):
        """Relinearised multiplies of one run: chains of t-1 = 2^16 squarings per candidate,
        s ANDs per candidate in paper mode, and the argmax circuit."""
        cands = 1 << self.s
        per_chain = (self.ctx.t - 1).bit_length() - 1 + bin(self.ctx.t - 1).count("1") - 1
        return self.n_classes * cands * (per_chain + (self.s if self.mode == PAPER else 0)) + self.circuit_muls

    def run(self, G_dev, W_dev, seed, keep=False):
        ctx = self.ctx
        N, L = ctx.N, ctx.L
        g = ctx.encrypt(G_dev, seed)                                           # tag ciphertexts
        rep = g.repeat(self.n_classes, 1, 1, 1)
        x = ctx.mul_plain(rep, W_dev.reshape(self.n_classes * self.n_tags, N))  # weighted tags
        x = x.view(self.n_classes, self.n_tags, 2, L, N)
        while x.shape[1] > 1:                                                  # sum over tags
            h = x.shape[1] // 2
            x = ctx.add(x[:, :h].contiguous(), x[:, h:].contiguous())
        scores = x.view(self.n_classes, 2, L, N)
        bits = ctx.mod_to_bits(scores, self.s, 0, (1 << self.s) - 1, self.mode)   # [s][3]
        self.circ.set_inputs(bits.transpose(0, 1).reshape(self.n_classes * self.s, 1, 2, L, N))
        self.circ.run()
        idx = self.circ.out(self.out_wires).view(2, 2, L, N)
        if keep:
            self.last = {"enc": g, "scores": scores, "bits": bits, "idx": idx}
        return ctx.decrypt(idx)                                                # [2][N] index bits


class FibonacciJob:
    """The data-oblivious Fibonacci of Listings 3 (bit-level) and 4 (bridged) over every slot.

    Slot j of batch entry b computes fibonacci(in[b, j]) for its own input.
    The initial values i = 0, a = 0, b = 1, r = 0 are fresh encryptions (E3
    encrypts the constants `_0_E`, `_1_M`), made with the input bits in one
    batched encrypt call; input wire w of batch entry b is ciphertext
    w * n + b of that call.
    """

    def __init__(self, ctx, kind, width=8, max_iter=10, n=1):
        assert kind in ("bits", "bridged")
        self.ctx, self.kind, self.width, self.max_iter, self.n = ctx, kind, width, max_iter, n
        net = circuits.Netlist(ctx.t)
        inp, i0 = net.inputs(width), net.inputs(width)
        if kind == "bits":
            a0, b0, r0 = (net.inputs(width) for _ in range(3))
            self.out_wires = net.fibonacci_bits(inp, i0, a0, b0, r0, max_iter)
            self.consts = [0] * (2 * width) + [1] + [0] * (2 * width - 1)      # i, a, b, r
        else:
            a0, b0, r0 = net.inputs(3)
            self.out_wires = [net.fibonacci_bridged(inp, i0, a0, b0, r0, max_iter)]
            self.consts = [0] * width + [0, 1, 0]
        self.net = net
        self.circ = circuits.Compiled(ctx, net, n)

    def input_slots(self, vals):
        """vals: device int64 [n][N] inputs -> slot values of every input wire [n_inputs][n][N].
        Without batching (t = 2) vals is [n][1] and each value sits in coefficient 0 of its
        plaintext polynomial (the other coefficients zero)."""
        import torch
        planes = torch.stack([(vals >> k) & 1 for k in range(self.width)])
        c = torch.tensor(self.consts, dtype=torch.int64, device=vals.device).view(-1, 1, 1)
        out = torch.cat([planes, c.expand(-1, vals.shape[0], vals.shape[1])])
        if not self.ctx.batching:
            poly = torch.zeros(out.shape[0], out.shape[1], self.ctx.N, dtype=torch.int64, device=vals.device)
            poly[:, :, :1] = out[:, :, :1]
            out = poly
        return out

    def set_inputs(self, vals, seed):
        slots = self.input_slots(vals).reshape(-1, self.ctx.N)
        enc = self.ctx.encrypt if self.ctx.batching else self.ctx.encrypt_poly
        cts = enc(slots, seed)
        self.circ.set_inputs(cts.view(-1, self.n, 2, self.ctx.L, self.ctx.N))

    def run(self):
        self.circ.run()

    def result(self):
        """[len(out)][n][2][L][N]: the bits of r (bit-level) or the single SecureMod r."""
        return self.circ.out(self.out_wires)

    def decrypt(self):
        """Decrypted r per slot: [n][N] (bits recombined for the bit-level program); without
        batching [n][1], coefficient 0."""
        out = self.result()
        if self.ctx.batching:
            d = [self.ctx.decrypt(out[k].contiguous()) for k in range(out.shape[0])]
        else:
            d = [self.ctx.decrypt_poly(out[k].contiguous())[:, :1] for k in range(out.shape[0])]
        if self.kind == "bridged":
            return d[0]
        return sum(dk << k for k, dk in enumerate(d))
