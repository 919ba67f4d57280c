"""File-level chunking (Sec. 3.11), on token ids (test infrastructure only).

The paper splits the input text into N roughly equal chunks at newline
boundaries and codes every chunk as an independent stream of one container
(Sec. 3.12).  Without the tokenizer this works on the token sequence: the
caller marks the ids that end a line (is_boundary[id] != 0), and

    target_k = ceil(k n / N)                      for k = 1 .. N - 1
    cut_k    = 1 + the first position p >= target_k - 1 whose token ends a line

so every chunk but the last ends with a line-ending token and holds about
n / N tokens.  A cut with no line end after its target, or at or before the
previous cut, is dropped; the chunks are tokens[cut_k .. cut_{k+1}) with
cut_0 = 0 and a last cut n.  Empty inputs give no chunk.
"""
from __future__ import annotations


def split_points(tokens, is_boundary, n_chunks: int) -> list[int]:
    """The cut positions 0 = c_0 < c_1 < ... < c_m = n (m chunks, m <= n_chunks)."""
    n = len(tokens)
    if n == 0:
        return [0]
    if n_chunks < 1:
        raise ValueError("n_chunks must be >= 1")
    cuts = [0]
    for k in range(1, n_chunks):
        target = -(-k * n // n_chunks)                 # ceil(k n / N)
        p = max(target - 1, 0)
        while p < n and not is_boundary[int(tokens[p])]:
            p += 1
        if p >= n:
            break                                      # no line end after the target
        c = p + 1
        if c > cuts[-1] and c < n:
            cuts.append(c)
    cuts.append(n)
    return cuts


def split(tokens, is_boundary, n_chunks: int):
    c = split_points(tokens, is_boundary, n_chunks)
    return [tokens[c[i]:c[i + 1]] for i in range(len(c) - 1)]
